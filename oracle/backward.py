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

In the identity-sketch mode with Omega = I the estimator equals the exact
leverage theta, whose gradient has the closed form 2 (I - H) W (A^+)^T.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from . import rng
from .estimator import count_sketch, gaussian_stage
from .linalg import pivoted_qr


def _copyltu(X: np.ndarray) -> np.ndarray:
    return np.tril(X) + np.tril(X, -1).T


def theta_fixed(A, perm, r, s, m, k, seed, sketch_identity=False, omega_identity=False):
    """theta~(A) with P and r fixed (the function whose gradient is taken)."""
    A = np.asarray(A, dtype=np.float64)
    cols = np.asarray(perm[:r])
    AK = A[:, cols]
    At = AK if sketch_identity else gaussian_stage(count_sketch(AK, s, seed), m, seed)
    qr = pivoted_qr(At, 0.0, forced_perm=np.arange(r), forced_rank=r)
    R11 = qr.R[:, :r]
    Om = np.eye(r) if omega_identity else rng.omega(r, k, seed)
    M = solve_triangular(R11, Om, lower=False)
    Y = AK @ M
    return np.sum(Y * Y, axis=1)


def gradient(A, w, perm, r, s, m, k, seed, sketch_identity=False, omega_identity=False):
    """dg/dA (n x d) for g = sum_i w_i theta~_i, FP64."""
    A = np.asarray(A, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    n, d = A.shape
    cols = np.asarray(perm[:r])
    AK = A[:, cols]
    At = AK if sketch_identity else gaussian_stage(count_sketch(AK, s, seed), m, seed)
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
        # G^T Xbar (s x r), then S^T: row i takes sigma_i * (G^T Xbar)[h(i), :]
        Gt = np.zeros((s, r))
        blk = 1 << 14
        for c0 in range(0, s, blk):
            c1 = min(s, c0 + blk)
            Gt[c0:c1] = rng.gaussian_sketch_block(m, s, seed, c0, c1).T @ Xbar
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
