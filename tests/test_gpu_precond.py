"""GPU parity of Alg. 11 (lev_precondition_dense / _csr) and of LSQR on A N (lev_lsqr_dense)
against the FP64 oracle (oracle/precond.py) and numpy's least squares.

* N: N N^T (unique, unlike N's signs) against the oracle's SVD of the same sketch (the GPU sketch
  read back: the SVD step alone), to 1e-8 of its largest entry; k equal.
* Theorem 8 (GSA preconditioning, Sec. 6.2) on the GPU's N: kappa(A N) <= xi eta (m = 4d, alpha = 0.3,
  eps = 1/2) for kappa(A) up to 1e6, with FP32 and split-BF16 sketches.
* LSQR: x against numpy's minimum-norm least squares. The passes round in FP32 (backward error
  about atol = 1e-6), so for b = A x0 + e with ||e|| = 1e-3 ||b|| the forward error is bounded
  by about atol kappa (1 + kappa ||r|| / (||A|| ||x||)); the tests take 20x that. The normal
  equations' residual ||A^T (A x - b)|| / (||A||_F ||A x - b||) is checked against
  1e-4 + 50 u_32 ||A|| ||x|| / ||A x - b||: A x is formed in FP32 in the passes, so the residual
  carries an absolute error of about u_32 ||A|| ||x||.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import estimator as E, precond as P

from ._gpu import lev_module, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    return lev_module()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle(0)


def _precond(L, h, A32, s, m, seed, tau, prec):
    import torch
    n, d = A32.shape
    dA = to_dev(A32)
    p = L.make_params(s=s, m=m, k=8, tau=tau, seed=seed, sketch_prec=prec)
    N = torch.empty((d, d), dtype=torch.float64, device="cuda")
    sig = torch.empty(d, dtype=torch.float64, device="cuda")
    k = L.lev_precondition_dense(h, dA, p, N, sigma=sig)
    At = torch.empty((m, d), device="cuda")
    L.lev_sketch_dense(h, dA, p, At)
    torch.cuda.synchronize()
    return dA, k, to_np(N), to_np(sig), to_np(At).astype(np.float64)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("r", [1e-2, 1e-6])
def test_preconditioner_matches_svd_and_bound(L, h, prec, r):
    n, d = 20000, 64
    A = W.fixed_svd(n, d, np.linspace(1.0, r, d), seed=3).astype(np.float32)
    s, m = 5 * (d * d + d), 4 * d
    dA, k, N, sig, At = _precond(L, h, A, s, m, 9, 1e-12, prec)
    _, s_ref, Vt = np.linalg.svd(At, full_matrices=False)
    assert k == d
    np.testing.assert_allclose(sig, s_ref, rtol=1e-9, atol=1e-12 * s_ref[0])
    Nr = Vt[:k].T / s_ref[:k][None, :]
    NN, NNr = N[:, :k] @ N[:, :k].T, Nr @ Nr.T
    assert np.abs(NN - NNr).max() <= 1e-8 * np.abs(NNr).max()
    assert np.all(N[:, k:] == 0)
    sv = np.linalg.svd(A.astype(np.float64) @ N[:, :k], compute_uv=False)
    assert sv[0] / sv[-1] <= P.kappa_bound(k, m, alpha=0.3, eps=0.5)


def _problem(n, d, kappa, seed, rank=None):
    rs = np.random.default_rng(seed)
    sig = np.geomspace(1.0, 1.0 / kappa, d)
    if rank is not None:
        sig[rank:] = 0.0
    A = W.fixed_svd(n, d, sig, seed=seed).astype(np.float32)
    x0 = rs.standard_normal(d)
    b = A.astype(np.float64) @ x0
    b = (b + 1e-3 * np.linalg.norm(b) / np.sqrt(n) * rs.standard_normal(n)).astype(np.float32)
    return A, b


def _check_solution(A, b, x, kappa, rcond=None):
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    want = np.linalg.lstsq(A64, b64, rcond=rcond)[0]
    r = A64 @ want - b64
    ratio = np.linalg.norm(r) / (np.linalg.norm(A64, 2) * np.linalg.norm(want))
    bound = 20 * 1e-6 * kappa * (1 + kappa * ratio)
    assert np.linalg.norm(x - want) <= bound * np.linalg.norm(want)
    rx = A64 @ x - b64
    floor = 50 * 2.0 ** -24 * np.linalg.norm(A64, 2) * np.linalg.norm(x) / np.linalg.norm(rx)
    assert np.linalg.norm(A64.T @ rx) <= (1e-4 + floor) * np.linalg.norm(A64) * np.linalg.norm(rx)


@pytest.mark.parametrize("n,d,kappa", [(100000, 64, 1e2), (200003, 256, 1e3), (50000, 77, 1e4)])
def test_lstsq_matches_numpy(L, h, n, d, kappa):
    A, b = _problem(n, d, kappa, seed=d)
    x, k, it, rn = L.lstsq(to_dev(A), to_dev(b), s=8 * d * 16, m=4 * d, seed=2, tau=1e-10, handle=h)
    assert k == d and 0 < it < 60
    _check_solution(A, b, to_np(x), kappa)
    assert L.lev_device_status(h) == 0


def test_iterations_do_not_grow_with_kappa(L, h):
    its = []
    for kappa in (1e2, 1e4, 1e6):
        A, b = _problem(60000, 48, kappa, seed=5)
        x, k, it, _ = L.lstsq(to_dev(A), to_dev(b), s=16384, m=192, seed=4, tau=1e-12, atol=1e-5, btol=1e-5, handle=h)
        its.append(it)
    assert max(its) <= 40 and max(its) - min(its) <= 10, its


def test_rank_deficient_and_padded_rows(L, h):
    import torch
    n, d, rank = 40000, 40, 25
    A, b = _problem(n, d, 1e2, seed=8, rank=rank)
    Ab = torch.zeros((n, 44), dtype=torch.float32, device="cuda")        # lda = 44, not a multiple of 4 in d
    Ab[:, :d] = to_dev(A)
    # tau above the split-BF16 sketch's noise floor (about 1e-5 sigma_1) and far below sigma_25 = 0.059
    x, k, it, _ = L.lstsq(Ab[:, :d], to_dev(b), s=8192, m=160, seed=1, tau=1e-4, handle=h)
    assert k == rank
    _check_solution(A, b, to_np(x), 1e2, rcond=1e-4)


def test_csr_preconditioner_bound(L, h):
    import torch
    n, d = 60000, 96
    C = W.csr_uniform(n, d, nnz_per_row=6, heavy_frac=0.01, heavy_nnz=48, seed=2)
    scale = np.exp(np.random.default_rng(0).standard_normal(d) * 2)          # column scaling: kappa ~ 1e3
    val = (C.val * scale[C.col]).astype(np.float32)
    p = L.make_params(s=16384, m=4 * d, k=8, tau=1e-12, seed=3, sketch_prec="bf16x3")
    N = torch.empty((d, d), dtype=torch.float64, device="cuda")
    k = L.lev_precondition_csr(h, to_dev(C.row_ptr), to_dev(C.col), to_dev(val), n, d, p, N)
    assert k == d
    Asp = sp.csr_matrix((val.astype(np.float64), C.col, C.row_ptr), shape=(n, d))
    assert np.linalg.cond(Asp.toarray()) > 50
    sv = np.linalg.svd(Asp @ to_np(N), compute_uv=False)
    assert sv[0] / sv[-1] <= P.kappa_bound(d, 4 * d, alpha=0.3, eps=0.5)


def test_lstsq_csr_matches_numpy(L, h):
    """Alg. 11 and LSQR on CSR input: rows of 0..40 entries (both pass kernels), scaled columns."""
    import torch
    rs = np.random.default_rng(6)
    n, d = 80000, 72
    lens = np.where(rs.random(n) < 0.05, rs.integers(9, 41, size=n), rs.integers(0, 9, size=n))
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = np.concatenate([rs.choice(d, size=l, replace=False) for l in lens]).astype(np.int32)
    scale = np.exp(rs.standard_normal(d))
    val = (rs.standard_normal(row_ptr[-1]) * scale[col]).astype(np.float32)
    Ad = sp.csr_matrix((val.astype(np.float64), col, row_ptr), shape=(n, d)).toarray()
    kappa = np.linalg.cond(Ad)
    x0 = rs.standard_normal(d)
    b = Ad @ x0
    b = (b + 1e-3 * np.linalg.norm(b) / np.sqrt(n) * rs.standard_normal(n)).astype(np.float32)
    dr, dc, dv = to_dev(row_ptr), to_dev(col), to_dev(val)
    p = L.make_params(s=16384, m=4 * d, k=8, tau=1e-10, seed=2, sketch_prec="bf16x3")
    N = torch.empty((d, d), dtype=torch.float64, device="cuda")
    k = L.lev_precondition_csr(h, dr, dc, dv, n, d, p, N)
    assert k == d
    x = torch.zeros(d, dtype=torch.float64, device="cuda")
    it, rn = L.lev_lsqr_csr(h, dr, dc, dv, n, d, N, k, to_dev(b), x)
    assert 0 < it < 60
    _check_solution(Ad.astype(np.float32), b, to_np(x), kappa)
