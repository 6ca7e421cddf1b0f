"""Oracle gradient of g(A) = sum_i w_i theta~_i(A) (FP64, numpy).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

The paper defines no backward pass; this is the adjoint of the estimator of
Alg. 10 (see ``oracle.estimator``) with the CountSketch S, the Gaussian G, the
JL matrix Omega, the pivot order P and the rank r held fixed:

  A~_K = G S A_K,  A~_K = Q_1 R_11 (Householder, diag(R_11) > 0),
  M = R_11^{-1} Omega,  Y = A_K M,  theta~_i = ||Y_i||^2.

Reverse mode, with W = diag(w):
  Z = 2 W Y;  C = A_K^T Z;  Rbar = -R_11^{-T} C M^T;
  Xbar = Q_1 copyltu(R_11 Rbar^T) R_11^{-T}   (QR adjoint with Qbar = 0,
         copyltu(X) = tril(X) + tril(X, -1)^T; Walter and Lehmann 2018);
  dg/dA_K = Z M^T + S^T G^T Xbar;  dg/dA = 0 on the columns outside K.

With the SRHT after the CountSketch (Sec. 3.4.2, 4.1), A~_K = G F S A_K with
F = sqrt(s/t) P H D (t x s) and G m x t, so the sketch term of the gradient is
S^T F^T G^T Xbar, F^T = D H P^T / sqrt(t) (H the unnormalised Walsh-Hadamard
matrix, symmetric; P^T scatters the t drawn rows, repeated draws adding up).

In the identity-sketch mode with Omega = I the estimator equals the exact
leverage theta, whose gradient has the closed form 2 (I - H) W (A^+)^T.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from . import rng
from .estimator import count_sketch, fwht, gaussian_stage, sketch
from .linalg import pivoted_qr


def _copyltu(X: np.ndarray) -> np.ndarray:
    return np.tril(X) + np.tril(X, -1).T


def theta_fixed(A, perm, r, s, m, k, seed, sketch_identity=False, omega_identity=False, srht_t=0):
    """theta~(A) with P and r fixed (the function whose gradient is taken)."""
    A = np.asarray(A, dtype=np.float64)
    cols = np.asarray(perm[:r])
    AK = A[:, cols]
    At = AK if sketch_identity else sketch(AK, s, m, seed, srht_t=srht_t)
    qr = pivoted_qr(At, 0.0, forced_perm=np.arange(r), forced_rank=r)
    R11 = qr.R[:, :r]
    Om = np.eye(r) if omega_identity else rng.omega(r, k, seed)
    M = solve_triangular(R11, Om, lower=False)
    Y = AK @ M
    return np.sum(Y * Y, axis=1)


def srht_adjoint(Tt: np.ndarray, s: int, seed: int) -> np.ndarray:
    """F^T Tt (s x r) for Tt (t x r): D H P^T Tt / sqrt(t), the adjoint of estimator.srht."""
    t = Tt.shape[0]
    X = np.zeros((s,) + Tt.shape[1:])
    np.add.at(X, rng.srht_rows(t, s, seed), Tt)
    return rng.srht_signs(s, seed)[:, None] * fwht(X) / np.sqrt(t)


def gradient(A, w, perm, r, s, m, k, seed, sketch_identity=False, omega_identity=False, srht_t=0):
    """dg/dA (n x d) for g = sum_i w_i theta~_i, FP64."""
    A = np.asarray(A, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    n, d = A.shape
    cols = np.asarray(perm[:r])
    AK = A[:, cols]
    At = AK if sketch_identity else sketch(AK, s, m, seed, srht_t=srht_t)
    qr = pivoted_qr(At, 0.0, forced_perm=np.arange(r), forced_rank=r)
    R11 = qr.R[:, :r]
    Q1 = qr.q_thin(r)
    Om = np.eye(r) if omega_identity else rng.omega(r, k, seed)
    M = solve_triangular(R11, Om, lower=False)
    Y = AK @ M
    Z = 2.0 * w[:, None] * Y
    C = AK.T @ Z
    Rbar = -solve_triangular(R11, C @ M.T, lower=False, trans="T")
    Xbar = solve_triangular(R11, (Q1 @ _copyltu(R11 @ Rbar.T)).T, lower=False).T
    if sketch_identity:
        T_rows = Xbar
    else:
        # G^T Xbar (s x r, or t x r after an SRHT, then F^T), then S^T: row i takes
        # sigma_i * (...)[h(i), :]
        cg = srht_t if srht_t else s
        Gt = np.zeros((cg, r))
        blk = 1 << 14
        for c0 in range(0, cg, blk):
            c1 = min(cg, c0 + blk)
            Gt[c0:c1] = rng.gaussian_sketch_block(m, cg, seed, c0, c1).T @ Xbar
        if srht_t:
            Gt = srht_adjoint(Gt, s, seed)
        b, sign = rng.bucket_and_sign(n, s, seed)
        T_rows = sign[:, None] * Gt[b]
    gK = Z @ M.T + T_rows
    g = np.zeros((n, d))
    g[:, cols] = gK
    return g


def exact_gradient(A, w):
    """Closed form 2 (I - H) W (A^+)^T of d/dA sum_i w_i theta_i(A) for full-column-rank A."""
    A = np.asarray(A, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    Ap = np.linalg.pinv(A)
    H = A @ Ap
    n = A.shape[0]
    return 2.0 * (np.eye(n) - H) @ (w[:, None] * Ap.T)
