"""GPU parity of the CountSketch + SRHT + Gaussian sketch (LEV_SKETCH_SRHT, Sec. 4.1) against
the FP64 oracle.

Sketch entries within c |G| |F| |S| |A| entrywise, where |F| = |H|/sqrt(t) has every entry
1/sqrt(t) (so |F| |S| |A| is the column sums of |S A| over sqrt(t) in every row); c = 3e-5 for the
FP32 Gaussian stage and 1e-4 for split BF16 (the FP32 butterflies add log2(s) roundings relative
to that scale, far below c). End to end: rank and pivots exact, theta within 1e-4.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import estimator as E, rng as orng

from ._gpu import lev_module, max_rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    return lev_module()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle(0)


def _srht_abs_scale(A64, s, m, t, seed):
    n, d = A64.shape
    b, _ = orng.bucket_and_sign(n, s, seed)
    Babs = np.zeros((s, d))
    np.add.at(Babs, b, np.abs(A64))
    Fabs = np.repeat(Babs.sum(axis=0, keepdims=True) / np.sqrt(t), t, axis=0)      # t x d
    return np.abs(orng.gaussian_sketch_block(m, t, seed, 0, t)) @ Fabs


@pytest.mark.parametrize("prec,c", [("fp32", 3e-5), ("bf16x3", 1e-4)])
@pytest.mark.parametrize("n,d,s,m,t", [(5000, 24, 1024, 96, 300), (20000, 64, 4096, 256, 1024), (700, 7, 1, 28, 1)])
def test_srht_sketch_parity(L, h, prec, c, n, d, s, m, t):
    import torch
    A = W.dense_heavy_rows(n, d, seed=n + d)
    p = L.make_params(s=s, m=m, k=8, seed=9, sketch_prec=prec, srht_t=t)
    At = torch.empty((m, d), device="cuda")
    L.lev_sketch_dense(h, to_dev(A), p, At)
    torch.cuda.synchronize()
    A64 = A.astype(np.float64)
    want = E.sketch(A64, s, m, 9, srht_t=t)
    scale = _srht_abs_scale(A64, s, m, t, 9)
    assert np.all(np.abs(to_np(At).astype(np.float64) - want) <= c * scale + 1e-30)


def test_srht_estimate_dense_matches_oracle(L, h):
    A = W.dense_lowrank_skewed(30000, 48, 30, seed=3)
    cfg = dict(s=8192, m=192, k=64, tau=1e-4, seed=5)
    theta, r, perm = L.estimate(to_dev(A), sketch_prec="bf16x3", final_prec="bf16x3", srht_t=2048, handle=h, **cfg)
    e = E.estimate(A.astype(np.float64), cfg["s"], cfg["m"], cfg["k"], cfg["tau"], cfg["seed"], srht_t=2048)
    assert r == e.rank == 30
    assert np.array_equal(to_np(perm)[:r], e.perm[:r])
    assert max_rel(to_np(theta), e.theta) <= 1e-4


def test_srht_estimate_csr_matches_oracle(L, h):
    import torch
    n, d = 40000, 96
    C = W.csr_uniform(n, d, nnz_per_row=6, heavy_frac=0.01, heavy_nnz=60, seed=4)
    cfg = dict(s=16384, m=384, k=64, tau=1e-5, seed=6)
    p = L.make_params(sketch_prec="bf16x3", srht_t=4096, **cfg)
    theta = torch.empty(n, device="cuda")
    r = L.lev_estimate_csr(h, to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val), n, d, p, theta)
    Asp = sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=(n, d))
    e = E.estimate(Asp, cfg["s"], cfg["m"], cfg["k"], cfg["tau"], cfg["seed"], srht_t=4096)
    assert r == e.rank == d
    assert max_rel(to_np(theta), e.theta) <= 1e-4


def test_srht_rejects_bad_sizes(L, h):
    """s not a power of two, or t > s: the sketch and the backward reject them (LEV_EINVAL)."""
    import torch
    A = to_dev(W.dense_gaussian(500, 8, 0).astype(np.float32))
    At = torch.empty((32, 8), device="cuda")
    for kw in [dict(s=1000, srht_t=100), dict(s=1024, srht_t=2048)]:
        with pytest.raises(L.LevError) as e:
            L.lev_sketch_dense(h, A, L.make_params(m=32, k=8, **kw), At)
        assert e.value.code == L.LEV_EINVAL
    p = L.make_params(s=1024, m=32, k=8, srht_t=256)
    _, st = L.forward_state(A, p, handle=h)
    g = torch.empty_like(A)
    bad = L.make_params(s=1024, m=32, k=8, srht_t=2048)
    with pytest.raises(L.LevError) as e:
        L.lev_backward_dense(h, A, bad, st["Atilde"], st["perm"], st["d_rank"], st["R"], st["Mfull"],
                             torch.ones(500, device="cuda"), g)
    assert e.value.code == L.LEV_EINVAL
