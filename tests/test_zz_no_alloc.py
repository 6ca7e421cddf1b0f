"""lev_rrqr_noalloc: the pivoted QR for callers that cannot call cudaMalloc.

Such callers (code inside another allocator's fixed memory budget, or on a
latency-critical path that cannot take cudaMalloc's implicit device
synchronisation) get the same factorisation from a fixed device scratch array.
This test calls it through the C ABI twice in a row and checks each result
against lev_rrqr (the allocating entry point) with the tolerances of the other
QR parity tests: pivots and rank identical, R within 1e-10 relative.
It sits in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from ._gpu import lev_module, to_dev, to_np

pytestmark = pytest.mark.gpu


def _sketch(m, d, r, seed):
    rs = np.random.default_rng(seed)
    X = rs.standard_normal((m, r)) @ rs.standard_normal((r, d))
    X *= np.exp(rs.standard_normal(d))[None, :]
    return X.astype(np.float32)


def _compare(L, h, m, d, r, tau, seed, want_rank=True):
    import torch
    At = to_dev(_sketch(m, d, r, seed=seed))
    perm_a = torch.empty(d, dtype=torch.int32, device="cuda")
    R_a = torch.empty((d, d), dtype=torch.float64, device="cuda")
    rank_a = L.lev_rrqr(h, At, tau, perm_a, R_a)
    perm_b = torch.full((d,), -1, dtype=torch.int32, device="cuda")
    R_b = torch.full((d, d), float("nan"), dtype=torch.float64, device="cuda")
    rank_b = L.lev_rrqr_noalloc(At, tau, perm_b, R_b, want_rank=want_rank)
    if not want_rank:
        # the call only enqueued its work: the rank is the number of nonzero rows of R
        torch.cuda.synchronize()
        rank_b = int(np.count_nonzero(np.diag(to_np(R_b))))
    assert rank_a == rank_b == r
    assert np.array_equal(to_np(perm_a), to_np(perm_b))
    Ra, Rb = to_np(R_a), to_np(R_b)
    assert np.max(np.abs(Ra - Rb)) <= 1e-10 * np.max(np.abs(Ra))


def test_rrqr_noalloc_matches_rrqr_twice():
    """Two calls in a row on the Gram route (d <= 1024, tau >= 1e-6), each against lev_rrqr."""
    L = lev_module()
    h = L.Handle(0)
    for call, (m, d, r, tau) in enumerate([(1024, 256, 200, 1e-4), (300, 64, 40, 1e-5)]):
        _compare(L, h, m, d, r, tau, seed=call)
    h.close()


def test_rrqr_noalloc_householder_route_and_no_rank_pointer():
    """tau < 1e-6 takes the Householder route through the same fixed array (a full-rank sketch, so
    the rank is exact at that threshold); then a call without a
    rank pointer (no synchronisation inside the call) on both routes."""
    L = lev_module()
    h = L.Handle(0)
    _compare(L, h, 300, 64, 64, 1e-7, seed=5)
    _compare(L, h, 300, 64, 64, 1e-7, seed=6, want_rank=False)
    _compare(L, h, 1024, 256, 200, 1e-4, seed=7, want_rank=False)
    h.close()


def test_rrqr_noalloc_rejects_oversized_shapes():
    import torch
    L = lev_module()
    At = torch.zeros((4096, 1024), dtype=torch.float32, device="cuda")
    perm = torch.empty(1024, dtype=torch.int32, device="cuda")
    R = torch.empty((1024, 1024), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LevError) as e:
        L.lev_rrqr_noalloc(At, 1e-5, perm, R)
    assert e.value.code == L.LEV_EINVAL
    assert "8 MiB" in str(e.value)
