"""Oracle of CountGauss preconditioning (Alg. 11) and of LSQR on the preconditioned problem (FP64).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

Alg. 11 (CountGaussPrecondition): A~ = G S A (Alg. 3), its SVD A~ = U Sigma V^T, the rank
k = #{sigma_j > zeta sigma_1} (the reading of step 3 in oracle/rank.py), N = V_{:, :k} Sigma_k^{-1}.
By Theorem 8 (GSA preconditioning, Sec. 6.2), kappa(A N) <= xi eta with high probability,
xi = (1 + a + sqrt(k/m)) / (1 - a - sqrt(k/m)), eta = (1 + eps) / (1 - eps), whatever kappa(A) is,
and N y^ = A^+ b for the minimum-length solution y^ of min_y ||A N y - b||.

LSQR (Paige and Saunders, ACM TOMS 8(1), 1982) on B = A N, written from the published
recurrences: Golub-Kahan bidiagonalisation beta_1 u_1 = b, alpha_1 v_1 = B^T u_1; then
beta_{i+1} u_{i+1} = B v_i - alpha_i u_i, alpha_{i+1} v_{i+1} = B^T u_{i+1} - beta_{i+1} v_i, and
the plane rotations that update y and the residual estimates (phibar = ||r||,
||B^T r|| = phibar alpha |c|). Readings: y_0 = 0; the iteration stops when
||B^T r|| <= atol ||B||_F-estimate ||r|| (the estimate being sqrt(sum of alpha_i^2 + beta_i^2)),
when ||r|| <= btol ||b||, or after max_iter steps.
"""
from __future__ import annotations

import numpy as np

from .estimator import sketch
from .rank import rank_svd


def precondition(A, s: int, m: int, seed: int, zeta: float, srht_t: int = 0):
    """Alg. 11: (N (d x k), k, sigma of the sketch)."""
    At = sketch(A, s, m, seed, srht_t)
    _, sig, Vt = np.linalg.svd(At, full_matrices=False)
    k = rank_svd(sig, zeta)
    N = Vt[:k].T / sig[:k][None, :]
    return N, k, sig


def kappa_bound(k: int, m: int, alpha: float, eps: float) -> float:
    """xi eta of Theorem 8 (GSA preconditioning, Sec. 6.2)."""
    q = np.sqrt(k / m)
    return (1 + alpha + q) / (1 - alpha - q) * (1 + eps) / (1 - eps)


def lsqr(A, b, N, max_iter: int = 1000, atol: float = 1e-14, btol: float = 1e-14, return_anorm: bool = False):
    """min_y ||A N y - b|| by LSQR (Paige and Saunders); returns (x = N y, y, iterations, ||r||
    estimate), and with ``return_anorm`` also the ||A N||_F estimate of the stopping rule."""
    A = np.asarray(A, dtype=np.float64) if not hasattr(A, "tocsr") else A.astype(np.float64)
    b = np.asarray(b, dtype=np.float64)
    B = lambda v: A @ (N @ v)
    Bt = lambda u: N.T @ (A.T @ u)
    y = np.zeros(N.shape[1])
    beta = np.linalg.norm(b)
    if beta == 0:
        return (N @ y, y, 0, 0.0) + ((0.0,) if return_anorm else ())
    u = b / beta
    v = Bt(u)
    alpha = np.linalg.norm(v)
    if alpha == 0:
        return (N @ y, y, 0, beta) + ((0.0,) if return_anorm else ())
    v = v / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    bnorm2 = alpha * alpha
    it = 0
    for it in range(1, max_iter + 1):
        u = B(v) - alpha * u
        beta = np.linalg.norm(u)
        if beta > 0:
            u = u / beta
        v = Bt(u) - beta * v
        alpha = np.linalg.norm(v)
        if alpha > 0:
            v = v / alpha
        bnorm2 += alpha * alpha + beta * beta
        rho = np.hypot(rhobar, beta)
        c, sn = rhobar / rho, beta / rho
        theta = sn * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = sn * phibar
        y = y + (phi / rho) * w
        w = v - (theta / rho) * w
        if phibar * alpha * abs(c) <= atol * np.sqrt(bnorm2) * phibar or phibar <= btol * np.linalg.norm(b):
            break
    return (N @ y, y, it, phibar) + ((float(np.sqrt(bnorm2)),) if return_anorm else ())
