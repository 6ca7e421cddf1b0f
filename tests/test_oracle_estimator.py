"""Pins for the oracle of Alg. 10 (CountGauss sketch -> pivoted QR -> JL row norms); no GPU."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import estimator as E, exact, rng


def test_count_sketch_equals_explicit_product():
    A = W.dense_gaussian(50, 3, 1)
    b, sign = rng.bucket_and_sign(50, 7, seed=4)
    S = np.zeros((7, 50))
    for i in range(50):                       # one +-1 per column of S (Sec. 3.4.3)
        S[b[i], i] = sign[i]
    np.testing.assert_allclose(E.count_sketch(A, 7, 4), S @ A, atol=1e-14)
    # row blocking does not change the result
    np.testing.assert_allclose(E.count_sketch(A, 7, 4, block=8), S @ A, atol=1e-14)


def test_count_sketch_csr_equals_dense():
    C = W.csr_uniform(300, 40, nnz_per_row=3, heavy_frac=0.05, heavy_nnz=20, seed=3)
    Asp = sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=C.shape)
    np.testing.assert_allclose(E.count_sketch(Asp, 64, 9), E.count_sketch(C.to_dense(), 64, 9),
                               atol=1e-12)


def test_gaussian_stage_equals_explicit_product():
    B = np.random.default_rng(0).standard_normal((300, 4))
    G = rng.gaussian_sketch_block(16, 300, 2, 0, 300)
    np.testing.assert_allclose(E.gaussian_stage(B, 16, 2, block=64), G @ B, atol=1e-12)


def test_identity_modes_reduce_to_exact_leverage():
    """S = I, G = I, Omega = I: theta~ is the exact leverage (Theorem 1, Sec. 2.2, equality case)."""
    A = W.dense_gaussian(400, 9, 2)
    th, r = exact.exact_leverage_qr(A, 1e-12)
    e = E.estimate(A, 0, 0, 0, 1e-12, 0, sketch_identity=True, omega_identity=True)
    assert e.rank == r == 9
    np.testing.assert_allclose(e.theta, th, atol=1e-12)


def test_rank_deficient_identity_mode_matches_leverage_of_A():
    rng_ = np.random.default_rng(4)
    A = rng_.standard_normal((300, 5)) @ rng_.standard_normal((5, 12))
    th, r = exact.exact_leverage_qr(A, 1e-10)
    e = E.estimate(A, 0, 0, 0, 1e-10, 0, sketch_identity=True, omega_identity=True)
    assert e.rank == r == 5
    np.testing.assert_allclose(e.theta, th, atol=1e-10)


def test_sketch_preserves_leverage_with_omega_identity():
    """Pi_1 = GS an OSE: theta~(Omega = I) within (1 +- eps)^-2 of theta (Sec. 3.3, Alg. 8)."""
    A = W.dense_gaussian(4000, 8, 3)
    th, _ = exact.exact_leverage_qr(A, 1e-12)
    d = 8
    e = E.estimate(A, 5 * (d * d + d) * 4, 16 * d, 0, 1e-12, 6, omega_identity=True)
    ratio = e.theta / th
    # (1 - eps)^2 <= sigma(GSU)^2 relative, eps = 0.5 gives a loose [0.44, 4] band
    assert ratio.min() > 1 / 4 and ratio.max() < 4
    assert abs(np.median(ratio) - 1) < 0.2


def test_jl_tail_per_row():
    """theta~_i / theta_i ~ chi^2_k / k when the sketch is exact; JL tail bound (Sec. 3.4.1)."""
    A = W.dense_gaussian(20000, 6, 7)
    th, _ = exact.exact_leverage_qr(A, 1e-12)
    k = 64
    e = E.estimate(A, 0, 0, k, 1e-12, 8, sketch_identity=True)
    ratio = e.theta / th
    assert abs(ratio.mean() - 1) < 5 * np.sqrt(2 / k) / np.sqrt(A.shape[0]) * 3
    for eps in (0.5, 0.8):
        frac = np.mean(np.abs(ratio - 1) > eps)
        bound = 2 * np.exp(-k * (eps ** 2 / 2 - eps ** 3 / 3) / 2)
        assert frac <= bound + 0.01, (eps, frac, bound)
    assert abs(e.theta.sum() - 6) < 5 * np.sqrt(2 * 6 / k) * 2


def test_full_estimator_small_dense():
    """The small dense workload: full rank 20, theta~ approximates theta (Sec. 6.2)."""
    cfg = W.CONFIGS["dense_2000x20_f64"]
    A = W.dense_gaussian(cfg["n"], cfg["d"], cfg["data_seed"])
    th, r = exact.exact_leverage_qr(A, cfg["tau"])
    e = E.estimate(A, cfg["s"], cfg["m"], cfg["k"], cfg["tau"], cfg["seed"])
    assert e.rank == r == 20
    assert sorted(e.perm) == list(range(20))
    ratio = e.theta / th
    assert abs(np.median(ratio) - 1) < 0.25
    assert e.theta.sum() == pytest.approx(20, rel=0.25)


def test_scale_invariance_is_exact():
    A = W.dense_gaussian(500, 6, 11)
    e1 = E.estimate(A, 200, 24, 16, 1e-12, 3)
    e2 = E.estimate(2.0 * A, 200, 24, 16, 1e-12, 3)
    assert np.array_equal(e1.perm, e2.perm)
    assert np.array_equal(e1.theta, e2.theta)


def test_duplicate_columns_reduce_rank():
    A = W.dense_gaussian(3000, 10, 12)
    A[:, 7] = 2.0 * A[:, 2]
    A[:, 9] = -0.5 * A[:, 4]
    e = E.estimate(A, 400, 40, 16, 1e-8, 5)
    assert e.rank == 8
    sel = set(e.perm[:8].tolist())
    assert not ({2, 7} <= sel) and not ({4, 9} <= sel)


def test_zero_rows_and_zero_matrix():
    A = W.dense_gaussian(200, 5, 13)
    A[[3, 50, 199]] = 0.0
    e = E.estimate(A, 64, 20, 8, 1e-10, 1)
    assert np.all(e.theta[[3, 50, 199]] == 0.0)
    z = E.estimate(np.zeros((50, 4)), 16, 8, 8, 1e-10, 1)
    assert z.rank == 0 and np.all(z.theta == 0)


def test_forced_pivots_reproduce():
    A = W.dense_gaussian(600, 7, 14)
    e = E.estimate(A, 128, 28, 16, 1e-10, 2)
    f = E.estimate(A, 128, 28, 16, 1e-10, 2, forced_perm=e.perm, forced_rank=e.rank)
    np.testing.assert_allclose(f.theta, e.theta, rtol=1e-12)
    np.testing.assert_allclose(f.R[:, :e.rank], e.R[:, :e.rank], rtol=1e-12, atol=1e-12)


def test_final_pass_equals_mfull_product():
    A = W.dense_gaussian(100, 6, 15)
    e = E.estimate(A, 64, 24, 10, 1e-10, 4)
    Mf = E.m_full(e.M, e.perm, 6)
    np.testing.assert_allclose(e.theta, np.sum((A @ Mf) ** 2, axis=1), rtol=1e-12)


def test_sketch_spectrum_bounds():
    """Lemma 5 (the spectrum of GSU, Sec. 4.2) with G scaled by 1/sqrt(m)."""
    n, k, m, s = 20000, 10, 200, 600
    U = np.linalg.qr(np.random.default_rng(1).standard_normal((n, k)))[0]
    sv = np.linalg.svd(E.sketch(U, s, m, 21), compute_uv=False)
    alpha, eps = 0.3, 0.5
    assert sv[0] < ((1 + alpha) + np.sqrt(k / m)) * (1 + eps)
    assert sv[-1] > ((1 - alpha) - np.sqrt(k / m)) * (1 - eps)


def test_back_substitution_and_omega_factor():
    """Step 6 (M = R_11^{-1} Omega, Alg. 8 step 4): a hand-solved 3 x 3 system, the residual
    R_11 M - Omega, and R_11^{-1} itself against the textbook inverse of a triangular matrix."""
    from oracle.linalg import back_substitute
    R = np.array([[2.0, 1.0, -1.0], [0.0, 4.0, 2.0], [0.0, 0.0, 0.5]])
    # x3 = 1 / 0.5 = 2; x2 = (8 - 2 x3) / 4 = 1; x1 = (1 - x2 + x3) / 2 = 1
    np.testing.assert_array_equal(back_substitute(R, np.array([[1.0], [8.0], [1.0]]))[:, 0], [1.0, 1.0, 2.0])
    rs = np.random.default_rng(5)
    R11 = np.triu(rs.standard_normal((40, 40))) + 8 * np.eye(40)
    M = E.omega_factor(R11, 12, seed=3)
    np.testing.assert_allclose(R11 @ M, rng.omega(40, 12, 3), atol=1e-13)
    assert M.shape == (40, 12)
    Minv = E.omega_factor(R11, 0, seed=3, omega_identity=True)
    np.testing.assert_allclose(Minv, np.linalg.inv(R11), atol=1e-13)
    assert np.all(np.tril(Minv, -1) == 0)                       # the inverse stays upper triangular
