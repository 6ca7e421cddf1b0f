"""Pins of the oracle's CountGauss preconditioner (Alg. 11) and LSQR (oracle/precond.py).

* Lemma 9 (the spectrum of AN, Sec. 6.2): the singular values of A N are those of (G S U)^+, U the
  left singular vectors of A, whatever Sigma is. With the seeded U of fixed_svd, A N therefore has
  the same singular values for kappa(A) = 1e2 and 1e8 (the linspace spectra of Sec. 7.3), and they
  equal 1 / sigma(G S U) computed directly from U.
* Theorem 8 (GSA preconditioning, Sec. 6.2): kappa(A N) <= xi eta (m = 4d, alpha = 0.3, eps = 1/2 for the
  CountSketch size 5 (d^2 + d) of Sec. 7.2).
* N y^ = A^+ b (the theorem's consistency part): against numpy's minimum-norm least squares, also
  for rank-deficient A (the tolerance zeta drops the zero singular values).
* LSQR: N = I on a well-conditioned problem equals numpy's least squares; preconditioning cuts the
  iterations on an ill-conditioned one.
"""
import numpy as np
import pytest

import workloads as W
from oracle import estimator as E, precond as P


def _linspace_A(n, d, r, seed=7):
    return W.fixed_svd(n, d, np.linspace(1.0, r, d), seed=seed)


def _U(n, d, seed=7):
    return W._haar_orthogonal(np.random.default_rng(seed), n, d)      # the U of fixed_svd


D, NROWS = 60, 6000
CFG = dict(s=5 * (D * D + D), m=4 * D, seed=5)


def test_spectrum_of_AN_is_that_of_GSU_inverse():
    U = _U(NROWS, D)
    s_gsu = np.linalg.svd(E.sketch(U, CFG["s"], CFG["m"], CFG["seed"]), compute_uv=False)
    want = np.sort(1.0 / s_gsu)[::-1]
    for r in (1e-2, 1e-5, 1e-8):
        A = _linspace_A(NROWS, D, r)
        N, k, _ = P.precondition(A, CFG["s"], CFG["m"], CFG["seed"], zeta=1e-12)
        assert k == D
        got = np.linalg.svd(A @ N, compute_uv=False)
        np.testing.assert_allclose(got, want, rtol=1e-6)


def test_kappa_bound():
    bound = P.kappa_bound(D, CFG["m"], alpha=0.3, eps=0.5)
    assert 26 < bound < 28
    for r in (1e-3, 1e-9):
        A = _linspace_A(NROWS, D, r, seed=11)
        N, k, _ = P.precondition(A, CFG["s"], CFG["m"], CFG["seed"], zeta=1e-14)
        s = np.linalg.svd(A @ N, compute_uv=False)
        assert s[0] / s[-1] <= bound
        assert np.linalg.cond(A) > 0.5 / r                       # while A itself is ill-conditioned


@pytest.mark.parametrize("rank", [D, 40])
def test_lsqr_on_AN_gives_the_pseudoinverse_solution(rank):
    sig = np.concatenate([np.linspace(1.0, 1e-4, rank), np.zeros(D - rank)])
    A = W.fixed_svd(NROWS, D, sig, seed=3)
    b = np.random.default_rng(1).standard_normal(NROWS)
    N, k, _ = P.precondition(A, CFG["s"], CFG["m"], CFG["seed"], zeta=1e-10)
    assert k == rank
    x, y, it, rnorm = P.lsqr(A, b, N, atol=1e-15, btol=1e-15)
    want = np.linalg.lstsq(A, b, rcond=1e-10)[0]
    np.testing.assert_allclose(x, want, rtol=0, atol=1e-9 * np.linalg.norm(want))
    assert it < 80
    np.testing.assert_allclose(rnorm, np.linalg.norm(A @ want - b), rtol=1e-8)


def test_lsqr_plain_and_iteration_counts():
    rs = np.random.default_rng(2)
    A = rs.standard_normal((500, 20))
    b = rs.standard_normal(500)
    x, _, _, _ = P.lsqr(A, b, np.eye(20))
    np.testing.assert_allclose(x, np.linalg.lstsq(A, b, rcond=None)[0], rtol=1e-10)
    A = _linspace_A(NROWS, D, 1e-4)
    b = rs.standard_normal(NROWS)
    N, _, _ = P.precondition(A, CFG["s"], CFG["m"], CFG["seed"], zeta=1e-12)
    it_pre = P.lsqr(A, b, N, atol=1e-10, btol=1e-10)[2]
    it_plain = P.lsqr(A, b, np.eye(D), atol=1e-10, btol=1e-10, max_iter=2000)[2]
    assert it_pre < 40 and it_plain > 3 * it_pre


def test_lsqr_norm_estimate_closed_form():
    """The ||A N||_F estimate of the stopping rule (Paige and Saunders): with orthonormal columns
    and N = I, LSQR ends after one step and A v_1 = alpha_1 u_1 + beta_2 u_2, so the estimate
    sqrt(alpha_1^2 + alpha_2^2 + beta_2^2) is ||A v_1|| = 1 (alpha_2 = 0)."""
    rs = np.random.default_rng(8)
    Q = np.linalg.qr(rs.standard_normal((300, 12)))[0]
    b = rs.standard_normal(300)
    x, y, it, rn, an = P.lsqr(Q, b, np.eye(12), atol=1e-12, btol=1e-12, return_anorm=True)
    assert it == 1
    assert abs(an - 1.0) < 1e-12
    np.testing.assert_allclose(x, Q.T @ b, atol=1e-12)
    np.testing.assert_allclose(rn, np.linalg.norm(b - Q @ (Q.T @ b)), rtol=1e-12)
