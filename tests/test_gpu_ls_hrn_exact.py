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


# ---- CSR A (lev_exact_csr): B = A_K^T A_K by the rows' outer products (Lemma 8, Sec. 5.1) ----

def _run_csr(L, h, C, **cfg):
    import torch
    n, d = C.shape
    p = L.make_params(sketch_prec="bf16x3", final_prec="fp32", **cfg)
    theta = torch.full((n,), float("nan"), device="cuda")
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    r = L.lev_exact_csr(h, to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val), n, d, p, theta, perm)
    torch.cuda.synchronize()
    return to_np(theta).astype(np.float64), r, to_np(perm)


def _scipy(C):
    import scipy.sparse as sp
    return sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=C.shape)


@pytest.mark.parametrize("n,d,heavy", [(60000, 96, 64), (7001, 33, 33)])
def test_csr_matches_oracle(L, h, n, d, heavy):
    C = W.csr_uniform(n, d, nnz_per_row=6, heavy_frac=0.02, heavy_nnz=heavy, seed=n % 97)
    cfg = dict(s=8192, m=4 * d, k=64, tau=1e-6, seed=5)
    th, r, perm = _run_csr(L, h, C, **cfg)
    want, k, operm = X.ls_hrn_exact(_scipy(C), cfg["s"], cfg["m"], cfg["tau"], cfg["seed"])
    assert r == k == d
    assert np.array_equal(perm[:r], operm[:k])
    assert max_rel(th, want) <= 1e-5
    assert abs(th.sum() - d) < 1e-5 * d                 # sum of exact leverage scores = rank
    assert L.lev_device_status(h) == 0


def test_csr_rank_deficient(L, h):
    n, d = 50000, 64
    C = W.csr_dup_columns(n, d, nnz_per_row=8, pairs=5, seed=8)
    cfg = dict(s=8192, m=256, k=64, tau=1e-5, seed=6)
    th, r, perm = _run_csr(L, h, C, **cfg)
    want, k, operm = X.ls_hrn_exact(_scipy(C), cfg["s"], cfg["m"], cfg["tau"], cfg["seed"])
    assert r == k == d - 5
    assert np.array_equal(perm[:r], operm[:k])
    assert max_rel(th, want) <= 1e-5
    assert abs(th.sum() - (d - 5)) < 1e-3


def test_csr_unsorted_duplicate_and_empty_rows(L, h):
    """Columns in any order, repeated columns (they add up), rows with no entries (theta = 0)."""
    rs = np.random.default_rng(12)
    n, d = 20000, 24
    lens = rs.integers(0, 9, size=n)
    lens[::97] = 0
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = rs.integers(0, d, size=row_ptr[-1]).astype(np.int32)           # unsorted, repeats
    val = rs.standard_normal(row_ptr[-1]).astype(np.float32)
    C = W.CSR(row_ptr, col, val, (n, d))
    cfg = dict(s=4096, m=96, k=32, tau=1e-6, seed=9)
    th, r, perm = _run_csr(L, h, C, **cfg)
    want, k, operm = X.ls_hrn_exact(_scipy(C), cfg["s"], cfg["m"], cfg["tau"], cfg["seed"])
    assert r == k == d
    assert np.array_equal(perm[:r], operm[:k])
    assert np.all(th[lens == 0] == 0)
    assert max_rel(th, want) <= 1e-5


def test_csr_repeat_runs_agree(L, h):
    """The FP64 atomic sums of B may round in another order each run: theta agrees to ~1e-12."""
    C = W.csr_uniform(30000, 48, nnz_per_row=6, heavy_frac=0.02, heavy_nnz=48, seed=3)
    cfg = dict(s=4096, m=192, k=32, tau=1e-6, seed=2)
    a, ra, pa = _run_csr(L, h, C, **cfg)
    b, rb, pb = _run_csr(L, h, C, **cfg)
    assert ra == rb and np.array_equal(pa, pb)
    assert max_rel(a, b) <= 1e-6
