"""Pins for the oracle gradient of sum_i w_i theta~_i (no GPU)."""
import numpy as np

import workloads as W
from oracle import backward as Bk, estimator as E

N, D, S, M_, K, SEED = 500, 8, 256, 32, 16, 7


def _setup():
    A = W.dense_heavy_rows(N, D, seed=3).astype(np.float64)
    w = W.uniform_weights(N, seed=4).astype(np.float64)
    e = E.estimate(A, S, M_, K, 1e-10, SEED)
    return A, w, e


def test_gradient_matches_central_finite_differences():
    A, w, e = _setup()
    g = Bk.gradient(A, w, e.perm, e.rank, S, M_, K, SEED)
    rs = np.random.default_rng(0)
    idx = [(int(i), int(j)) for i, j in zip(rs.integers(0, N, 60), rs.integers(0, D, 60))]
    # include the heavy rows, where the gradient is largest
    heavy = np.nonzero(np.abs(A).max(axis=1) > 20)[0][:5]
    idx += [(int(i), j) for i in heavy for j in range(D)]
    scale = np.abs(g).max()
    for i, j in idx:
        h = 1e-6 * max(1.0, abs(A[i, j]))
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (w @ Bk.theta_fixed(Ap, e.perm, e.rank, S, M_, K, SEED)
              - w @ Bk.theta_fixed(Am, e.perm, e.rank, S, M_, K, SEED)) / (2 * h)
        assert abs(fd - g[i, j]) <= 1e-6 * scale + 1e-5 * abs(fd), (i, j, fd, g[i, j])


def test_theta_fixed_equals_estimator():
    A, w, e = _setup()
    np.testing.assert_allclose(Bk.theta_fixed(A, e.perm, e.rank, S, M_, K, SEED), e.theta, rtol=1e-10)


def test_identity_mode_gradient_is_exact_closed_form():
    """Identity sketch, Omega = I: theta~ = theta and the gradient is 2 (I - H) W (A^+)^T."""
    A, w, _ = _setup()
    g = Bk.gradient(A, w, np.arange(D), D, 0, 0, 0, 0, sketch_identity=True, omega_identity=True)
    ge = Bk.exact_gradient(A, w)
    assert np.abs(g - ge).max() <= 1e-10 * np.abs(ge).max()


def test_gradient_zero_outside_selected_columns():
    A, w, _ = _setup()
    A = A.copy()
    A[:, 5] = 3.0 * A[:, 1]
    e = E.estimate(A, S, M_, K, 1e-8, SEED)
    assert e.rank == D - 1
    g = Bk.gradient(A, w, e.perm, e.rank, S, M_, K, SEED)
    dropped = e.perm[e.rank:]
    assert np.all(g[:, dropped] == 0)


def _setup_srht(t=64):
    A = W.dense_heavy_rows(N, D, seed=3).astype(np.float64)
    w = W.uniform_weights(N, seed=4).astype(np.float64)
    e = E.estimate(A, S, M_, K, 1e-10, SEED, srht_t=t)
    return A, w, e


def test_srht_adjoint_is_the_transpose_of_the_srht():
    """<F B, Y> = <B, F^T Y> for random B (s x 3) and Y (t x 3), with repeated row draws (t = s)."""
    rs = np.random.default_rng(5)
    for t in (16, S):
        B = rs.standard_normal((S, 3))
        Y = rs.standard_normal((t, 3))
        lhs = np.sum(E.srht(B, t, SEED) * Y)
        rhs = np.sum(B * Bk.srht_adjoint(Y, S, SEED))
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


def test_srht_gradient_matches_central_finite_differences():
    A, w, e = _setup_srht()
    np.testing.assert_allclose(Bk.theta_fixed(A, e.perm, e.rank, S, M_, K, SEED, srht_t=64), e.theta, rtol=1e-10)
    g = Bk.gradient(A, w, e.perm, e.rank, S, M_, K, SEED, srht_t=64)
    rs = np.random.default_rng(1)
    idx = [(int(i), int(j)) for i, j in zip(rs.integers(0, N, 40), rs.integers(0, D, 40))]
    heavy = np.nonzero(np.abs(A).max(axis=1) > 20)[0][:3]
    idx += [(int(i), j) for i in heavy for j in range(D)]
    scale = np.abs(g).max()
    for i, j in idx:
        h = 1e-6 * max(1.0, abs(A[i, j]))
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (w @ Bk.theta_fixed(Ap, e.perm, e.rank, S, M_, K, SEED, srht_t=64)
              - w @ Bk.theta_fixed(Am, e.perm, e.rank, S, M_, K, SEED, srht_t=64)) / (2 * h)
        assert abs(fd - g[i, j]) <= 1e-6 * scale + 1e-5 * abs(fd), (i, j, fd, g[i, j])

