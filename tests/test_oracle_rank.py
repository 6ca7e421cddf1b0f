"""Pins of the oracle's SVD rank rule and strong-RRQR swaps (oracle/rank.py).

* SVD rank: matrices with known singular values (fixed_svd, Sec. 7.1's table: 15 ones, 15 at
  1e-6, 30 at 1e-7; and 15 ones, 15 at 1e-3, 30 at 4e-5) give the rank the table and Sec. 7.4
  state at the paper's cutoffs (10^-6.5 and 2e-4), on A and on its CountGauss sketch (Lemma on the
  spectrum of GSA: the sketch keeps each singular value within a constant factor, far inside a
  gap of 10).
* Strong RRQR: the Kahan matrix (the textbook matrix on which QR in its natural column order hides
  the rank: |r_nn| is hundreds of times sigma_n) breaks the SRRQR bound in that order and meets
  every SRRQR inequality after the swaps; each swap multiplies |det R11| by exactly its rho
  (Gu and Eisenstat's determinant identity); the bounds hold on random matrices with a gap.
"""
import numpy as np
import pytest

import workloads as W
from oracle import estimator as E, rank as K
from oracle.linalg import pivoted_qr


def _kahan(n, c=0.285):
    s = np.sqrt(1 - c * c)
    return np.diag(s ** np.arange(n)) @ (np.eye(n) + np.triu(-c * np.ones((n, n)), 1))


def _bounds_hold(A, perm, k, phi, slack=1.0 + 1e-9):
    R = K.r_factor(A, perm)
    d = A.shape[1]
    sA = K.singular_values(A)
    f = np.sqrt(1 + phi * phi * k * (d - k))
    s11 = K.singular_values(R[:k, :k])
    s22 = K.singular_values(R[k:, k:]) if k < d else np.zeros(0)
    rho, X, gamma, inv_omega = K.srrqr_measures(R, k)
    return (np.all(s11 * f * slack >= sA[:k]) and np.all(s22 <= sA[k:k + s22.size] * f * slack)
            and np.all(np.abs(X) <= phi * slack) and np.all(gamma[None, :] * inv_omega[:, None] <= phi * slack))


@pytest.mark.parametrize("sig_small,sig_tail,zeta", [(1e-6, 1e-7, 10 ** -6.5), (1e-3, 4e-5, 2e-4)])
def test_svd_rank_of_fixed_spectra(sig_small, sig_tail, zeta):
    sig = np.concatenate([np.ones(15), np.full(15, sig_small), np.full(30, sig_tail)])
    A = W.fixed_svd(3000, 60, sig, seed=7)
    sA = K.singular_values(A)
    np.testing.assert_allclose(sA, sig, rtol=1e-6, atol=1e-14)
    assert K.rank_svd(sA, zeta) == 30
    At = E.sketch(A, s=5 * (60 * 60 + 60), m=120, seed=3)
    assert K.rank_svd(K.singular_values(At), zeta) == 30
    assert K.rank_svd(np.zeros(5), 0.1) == 0


def test_kahan_needs_swaps_and_then_meets_every_bound():
    n, phi = 30, 2.0
    A = _kahan(n)
    k = n - 1
    assert not _bounds_hold(A, np.arange(n), k, phi)          # natural order: |r_nn| >> sigma_n
    perm, rhos, dets = K.srrqr(A, k, phi, np.arange(n))
    assert len(rhos) >= 1 and sorted(perm.tolist()) == list(range(n))
    assert _bounds_hold(A, perm, k, phi)
    R = K.r_factor(A, perm)
    assert abs(R[k, k]) <= K.singular_values(A)[k] * np.sqrt(1 + phi * phi * k)


def test_each_swap_scales_det_by_its_rho():
    rs = np.random.default_rng(4)
    A = rs.standard_normal((80, 24)) @ np.diag(np.logspace(0, -6, 24)) @ rs.standard_normal((24, 24))
    k, phi = 12, 1.01
    perm, rhos, dets = K.srrqr(A, k, phi, rs.permutation(24))
    assert len(rhos) >= 2
    for t, r in enumerate(rhos):
        assert r > phi
        np.testing.assert_allclose(dets[t + 1] / dets[t], r, rtol=1e-8)
    assert _bounds_hold(A, perm, k, phi)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bounds_on_random_matrices_with_a_gap(seed):
    rs = np.random.default_rng(seed)
    d, k = 40, 25
    sig = np.concatenate([np.logspace(0, -2, k), np.logspace(-7, -9, d - k)])
    A = W.fixed_svd(500, d, sig, seed=seed + 10)
    qr = pivoted_qr(A, 0.0)
    perm, rhos, dets = K.srrqr(A, k, 2.0, qr.perm)
    assert _bounds_hold(A, perm, k, 2.0)
    assert all(b > a for a, b in zip(dets[:-1], dets[1:]))


def test_measures_against_definitions():
    """rho from explicit inverses and norms on a small matrix (no back-substitution)."""
    rs = np.random.default_rng(9)
    A = rs.standard_normal((9, 6))
    perm = np.array([3, 0, 5, 1, 4, 2])
    k = 3
    R = K.r_factor(A, perm)
    Q, R2 = np.linalg.qr(A[:, perm])
    assert np.allclose(np.abs(R), np.abs(R2))
    inv = np.linalg.inv(R[:k, :k])
    rho, X, gamma, inv_omega = K.srrqr_measures(R, k)
    np.testing.assert_allclose(X, inv @ R[:k, k:], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(inv_omega, np.linalg.norm(inv, axis=1), rtol=1e-12)
    np.testing.assert_allclose(gamma, np.linalg.norm(R[k:, k:], axis=0), rtol=1e-12)
    for i in range(k):
        for j in range(6 - k):
            assert abs(rho[i, j] ** 2 - (X[i, j] ** 2 + (gamma[j] * inv_omega[i]) ** 2)) < 1e-10


def test_estimate_with_svd_rank_on_fixed_svd_2_5e4():
    """Sec. 7.4's case: fixed_svd_2.5e4 with the cutoff 2e-4 has numerical rank 30; the estimate
    with the SVD rule finds it, and equals the forced-pivot estimate at those columns."""
    sig = np.concatenate([np.ones(15), np.full(15, 1e-3), np.full(30, 4e-5)])
    A = W.fixed_svd(4000, 60, sig, seed=7)
    cfg = dict(s=4096, m=120, k=64, tau=2e-4, seed=5)
    e = E.estimate(A, rank_rule="svd", **cfg)
    assert e.rank == 30
    f = E.estimate(A, forced_perm=e.perm, forced_rank=30, **cfg)
    np.testing.assert_array_equal(e.theta, f.theta)
    g = E.estimate(A, rank_rule="svd", srrqr_phi=2.0, **cfg)
    assert g.rank == 30
    R = K.r_factor(g.Atilde, g.perm)
    rho = K.srrqr_measures(R, 30)[0]
    assert rho.max() <= 2.0


def test_r_factor_has_a_nonnegative_diagonal():
    """R of the QR at a column order, normalised to diag(R) >= 0: numpy's R up to row signs."""
    rs = np.random.default_rng(12)
    X = rs.standard_normal((40, 9))
    perm = rs.permutation(9)
    R = K.r_factor(X, perm)
    assert np.all(np.diag(R) >= 0)
    np.testing.assert_allclose(np.abs(R), np.abs(np.linalg.qr(X[:, perm], mode="r")), atol=1e-12)
    np.testing.assert_allclose(R.T @ R, X[:, perm].T @ X[:, perm], atol=1e-10)


def test_estimate_takes_srrqr_swaps_at_the_svd_rank():
    """Alg. 10 with the SVD rank rule and strong RRQR (identity sketch, so A~ = A): on the Kahan
    matrix the SVD rule gives k = n - 1; at phi = 1.05 the greedy pivoted order breaks the SRRQR
    bounds there, and the estimate's columns are the swaps at that k from that order, which meet
    every bound."""
    n, phi = 30, 1.05
    A = _kahan(n)
    sA = K.singular_values(A)
    zeta = 10 * sA[-1] / sA[0]
    assert sA[-2] > zeta * sA[0]
    greedy = pivoted_qr(A, 0.0).perm
    assert not _bounds_hold(A, greedy, n - 1, phi)
    e = E.estimate(A, 0, 0, 0, zeta, 0, sketch_identity=True, omega_identity=True, rank_rule="svd",
                   srrqr_phi=phi)
    assert e.rank == n - 1
    assert _bounds_hold(A, e.perm, n - 1, phi)
    assert np.array_equal(e.perm, K.srrqr(A, n - 1, phi, greedy)[0])


def test_estimate_srrqr_uses_the_rank_it_found():
    """The swaps run at the rank the SVD rule finds (k = 8 of 12 on a seeded rank-8 matrix with
    noise 1e-10): at phi = 1.0001 they pick a different column set than swaps at k - 1 would, and
    the result is the strong-RRQR order at k from the greedy start."""
    rs = np.random.default_rng(3)
    U = np.linalg.qr(rs.standard_normal((200, 8)))[0]
    A = U @ np.diag(np.logspace(0, -2, 8)) @ rs.standard_normal((8, 12)) + 1e-10 * rs.standard_normal((200, 12))
    phi = 1.0001
    e = E.estimate(A, 0, 0, 0, 1e-6, 0, sketch_identity=True, omega_identity=True, rank_rule="svd",
                   srrqr_phi=phi)
    assert e.rank == 8
    greedy = pivoted_qr(A, 0.0).perm
    want = K.srrqr(A, 8, phi, greedy)[0]
    assert np.array_equal(e.perm, want)
    assert set(want[:8].tolist()) != set(K.srrqr(A, 7, phi, greedy)[0][:8].tolist())
    assert K.srrqr_measures(K.r_factor(A, e.perm), 8)[0].max() <= phi
