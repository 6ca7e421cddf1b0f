"""GPU parity of Alg. 7 (LS-HRN-exact, lev_exact_dense) against the FP64 oracle.

Rank and pivots bit-exact; theta within 1e-5 relative per row with the FP32 final pass and
5e-5 with the split-BF16 one (the FP64 Gram matrix and Cholesky are far more accurate than the
FP32 cast of R^{-1} and the final pass).
"""
import numpy as np
import pytest

import workloads as W
from oracle import exact as X

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


def _run(L, h, A, final_prec, **cfg):
    import torch
    n, d = A.shape
    p = L.make_params(sketch_prec="bf16x3", final_prec=final_prec, **cfg)
    theta = torch.full((n,), float("nan"), device="cuda")
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    r = L.lev_exact_dense(h, to_dev(A), p, theta, perm)
    torch.cuda.synchronize()
    return to_np(theta).astype(np.float64), r, to_np(perm)


@pytest.mark.parametrize("final_prec,tol", [("fp32", 1e-5), ("bf16x3", 5e-5)])
def test_full_rank_matches_oracle_and_exact(L, h, final_prec, tol):
    A = W.dense_heavy_rows(3000, 20, seed=21)
    cfg = dict(s=1024, m=80, k=64, tau=1e-8, seed=3)
    th, r, perm = _run(L, h, A, final_prec, **cfg)
    want, k, operm = X.ls_hrn_exact(A.astype(np.float64), cfg["s"], cfg["m"], cfg["tau"], cfg["seed"])
    assert r == k == 20
    assert np.array_equal(perm[:r], operm[:k])
    assert max_rel(th, want) <= tol
    ex, _ = X.exact_leverage_qr(A.astype(np.float64), 1e-10)          # the rank is found: exact scores
    assert max_rel(th, ex) <= tol
    assert L.lev_device_status(h) == 0


def test_rank_deficient(L, h):
    A = W.dense_heavy_rows(4000, 12, seed=5)
    A[:, 9] = 2.0 * A[:, 4]
    cfg = dict(s=2048, m=48, k=32, tau=1e-5, seed=2)
    th, r, perm = _run(L, h, A, "fp32", **cfg)
    want, k, operm = X.ls_hrn_exact(A.astype(np.float64), cfg["s"], cfg["m"], cfg["tau"], cfg["seed"])
    assert r == k == 11
    assert np.array_equal(perm[:r], operm[:k])
    assert not ({4, 9} <= set(perm[:r].tolist()))
    assert max_rel(th, want) <= 1e-5
    assert abs(th.sum() - 11) < 1e-3


@pytest.mark.parametrize("n,d,rank,lda", [(20000, 64, 40, 64), (5000, 37, 30, 41)])
def test_low_rank_skewed_and_strided(L, h, n, d, rank, lda):
    import torch
    A = W.dense_lowrank_skewed(n, d, rank, seed=4)
    cfg = dict(s=8192, m=4 * d, k=64, tau=1e-4, seed=7)
    p = L.make_params(sketch_prec="bf16x3", final_prec="bf16x3", **cfg)
    Ab = torch.zeros((n, lda), dtype=torch.float32, device="cuda")
    Ab[:, :d] = to_dev(A)
    theta = torch.empty(n, device="cuda")
    r = L.lev_exact_dense(h, Ab[:, :d], p, theta)
    torch.cuda.synchronize()
    want, k, _ = X.ls_hrn_exact(A.astype(np.float64), cfg["s"], cfg["m"], cfg["tau"], cfg["seed"])
    assert r == k == rank
    assert max_rel(to_np(theta).astype(np.float64), want) <= 5e-5


def test_rejects_unsupported(L, h):
    import torch
    p = L.make_params(s=64, m=8, k=4, omega_identity=True)
    with pytest.raises(L.LevError) as e:
        L.lev_exact_dense(h, torch.zeros((10, 4), device="cuda"), p, torch.empty(10, device="cuda"))
    assert e.value.code == L.LEV_EINVAL
