"""lev_exact_reference_*: exact leverage scores of A itself (Sec. 1 definition, Alg. 5's Gram route
with the QR orthogonaliser) against the FP64 oracle's two exact routes.

Tolerances: the Gram matrix of FP32 data is formed to about FP64 accuracy and factored in FP64, so
R carries a relative error of about u_64 kappa(A_K)^2; theta_i = ||A_{i,K} R^{-1}||^2 is then summed
by the FP32 final pass (a relative error of a few u_32 times the row's amplification), so theta is
held to 1e-4 relative, the bar of the FP32 path. The pivots are those of the column-pivoted QR of A
(greatest trailing norm, ties to the lowest index) and are compared bit for bit on the first r
positions, as in the QR parity tests.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import exact as X, linalg as OL

from ._gpu import lev_module, max_rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lev_module()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle(0)


@pytest.mark.parametrize("n,d,rank,tau", [(3000, 40, 40, 1e-5), (20000, 64, 40, 1e-4), (65536, 256, 200, 1e-4),
                                          (1, 1, 1, 1e-5), (777, 130, 130, 1e-5)])
def test_exact_reference_dense(L, h, n, d, rank, tau):
    import torch
    if rank == d:
        A = W.dense_gaussian(n, d, seed=n + d).astype(np.float32)
    else:
        A = W.dense_lowrank_skewed(n, d, rank, seed=n + d)
    A64 = A.astype(np.float64)
    theta = torch.empty(n, device="cuda")
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    r = L.lev_exact_reference_dense(h, to_dev(A), tau, theta, perm)
    want, k = X.exact_leverage_gram(A64, tau)
    assert r == k == rank
    got = to_np(theta).astype(np.float64)
    assert max_rel(got, want) <= 1e-4
    if n >= d:
        w2, k2 = X.exact_leverage_qr(A64, tau)
        assert k2 == rank and max_rel(got, w2) <= 1e-4
    q = OL.pivoted_qr(A64, tau)
    assert np.array_equal(to_np(perm)[:r], q.perm[:r])
    assert abs(got.sum() - rank) <= 1e-4 * rank
    assert np.all(got >= 0) and np.all(got <= 1 + 1e-4)


def test_exact_reference_csr(L, h):
    import torch
    C = W.csr_uniform(40000, 128, nnz_per_row=8, heavy_frac=0.01, heavy_nnz=64, seed=6)
    n, d = C.shape
    theta = torch.empty(n, device="cuda")
    r = L.lev_exact_reference_csr(h, to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val), n, d, 1e-5, theta)
    A = sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=(n, d))
    want, k = X.exact_leverage_gram(A, 1e-5)
    assert r == k == d
    got = to_np(theta).astype(np.float64)
    assert max_rel(got, want) <= 1e-4
    assert abs(got.sum() - d) <= 1e-3


def test_exact_reference_rank_zero_and_rejections(L, h):
    import torch
    A = torch.zeros((500, 8), device="cuda")
    theta = torch.full((500,), 7.0, device="cuda")
    assert L.lev_exact_reference_dense(h, A, 1e-5, theta) == 0
    assert torch.all(theta == 0)
    with pytest.raises(L.LevError) as e:
        L.lev_exact_reference_dense(h, A, 1e-8, theta)
    assert e.value.code == L.LEV_EINVAL
    with pytest.raises(L.LevError) as e:
        L.lev_exact_reference_dense(h, torch.zeros((10, 1100), device="cuda"), 1e-5, torch.empty(10, device="cuda"))
    assert e.value.code == L.LEV_EINVAL
    assert L.lev_device_status(h) == 0
