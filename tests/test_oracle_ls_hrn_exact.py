"""Pins for the oracle's Alg. 7 (LS-HRN-exact), no GPU.

When the sketch's pivoted QR finds the rank of A, range(A_K) = range(A) and the scores equal the
exact leverage scores of A (the statement after Alg. 7: if k = rank(A) then theta~ = theta(A_k)).
These pins check that against the pseudo-inverse definition, against an independent solve of
a_K B^{-1} a_K^T, and dense against CSR.
"""
import numpy as np
import scipy.sparse as sp

import workloads as W
from oracle import exact


def brute_force_leverage(A):
    """diag(A (A^T A)^+ A^T) with numpy's SVD pseudo-inverse (Sec. 1, eq. (1))."""
    return np.diag(A @ np.linalg.pinv(A.T @ A) @ A.T)


def test_full_rank_equals_exact_leverage():
    A = W.dense_gaussian(300, 12, 3).astype(np.float64)
    A *= np.exp(np.random.default_rng(3).standard_normal(12))[None, :]
    th, k, perm = exact.ls_hrn_exact(A, s=128, m=48, tau=1e-10, seed=5)
    assert k == 12
    assert sorted(perm.tolist()) == list(range(12))
    np.testing.assert_allclose(th, brute_force_leverage(A), rtol=0, atol=1e-10)


def test_rank_deficient_equals_exact_leverage_of_a():
    rs = np.random.default_rng(7)
    A = rs.standard_normal((400, 5)) @ rs.standard_normal((5, 12))       # rank 5, 12 columns
    th, k, perm = exact.ls_hrn_exact(A, s=256, m=48, tau=1e-8, seed=2)
    assert k == 5
    np.testing.assert_allclose(th, brute_force_leverage(A), rtol=0, atol=1e-9)
    assert abs(th.sum() - 5) < 1e-9
    assert np.all(th >= -1e-12) and np.all(th <= 1 + 1e-12)


def test_equals_direct_solve_on_the_selected_columns():
    """theta_i = a_{i,K} B^{-1} a_{i,K}^T with B = A_K^T A_K, by a linear solve (no eigenvectors)."""
    A = W.dense_heavy_rows(500, 9, seed=4).astype(np.float64)
    th, k, perm = exact.ls_hrn_exact(A, s=256, m=36, tau=1e-10, seed=9)
    AK = A[:, perm[:k]]
    B = AK.T @ AK
    want = np.einsum("ij,ji->i", AK, np.linalg.solve(B, AK.T))
    np.testing.assert_allclose(th, want, rtol=1e-10, atol=1e-13)


def test_csr_equals_dense():
    C = W.csr_uniform(2000, 40, nnz_per_row=6, heavy_frac=0.02, heavy_nnz=30, seed=3)
    Asp = sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=(2000, 40))
    t_sp, k_sp, p_sp = exact.ls_hrn_exact(Asp, s=512, m=160, tau=1e-10, seed=1)
    t_de, k_de, p_de = exact.ls_hrn_exact(Asp.toarray(), s=512, m=160, tau=1e-10, seed=1)
    assert k_sp == k_de and np.array_equal(p_sp, p_de)
    np.testing.assert_allclose(t_sp, t_de, rtol=1e-12, atol=1e-14)


def test_identity_sketch_selects_by_the_qr_of_a():
    A = W.dense_gaussian(200, 10, 1).astype(np.float64)
    A[:, 7] = 3.0 * A[:, 2]
    th, k, perm = exact.ls_hrn_exact(A, s=0, m=0, tau=1e-9, seed=0, sketch_identity=True)
    assert k == 9
    assert not ({2, 7} <= set(perm[:k].tolist()))
    np.testing.assert_allclose(th, brute_force_leverage(A), rtol=0, atol=1e-9)
