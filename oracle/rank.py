"""Oracle rank decisions beyond the diagonal test of the pivoted QR (FP64, numpy).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

* SVD rank (Alg. 11 step 3, and Sec. 7.2: where the |R_kk| < c |R_11| test of the pivoted QR
  misses a small gap, as on fixed_svd_1e7, the rank is better read off the singular values and
  the pivoted QR kept only for the column order): k = #{j : sigma_j > zeta sigma_1}.
  Reading: Alg. 11 writes an argmax over the set {sigma_j : sigma_j / sigma_1 <= zeta}, which taken
  literally picks the small singular values; the tolerance on rcond it describes is the count of
  singular values above zeta sigma_1, which is what is computed here.
* Strong RRQR at a fixed k (Def. of SRRQR and Alg. 2, after Gu and Eisenstat's swap algorithm):
  for the column order P, with A P = Q R and R = [[R11, R12], [0, R22]] (R11 k x k),
      rho_ij = sqrt( ((R11^{-1} R12)_ij)^2 + (gamma_j(R22) / omega_i(R11))^2 ),
  gamma_j = ||R22 e_j|| (column norms), omega_i = 1 / ||e_i^T R11^{-1}|| (row norms of the
  inverse). While max rho_ij > phi, column i of the selected set and column k + j of the rest
  trade places; each swap multiplies |det R11| by rho_ij > phi, so the loop ends. At the end
  |(R11^{-1} R12)_ij| <= phi, gamma_j / omega_i <= phi, and the singular-value bounds
      sigma_i(R11) >= sigma_i(A) / sqrt(1 + phi^2 k (d - k)),
      sigma_j(R22) <= sigma_{k+j}(A) sqrt(1 + phi^2 k (d - k))
  hold. Readings: the pair with the largest rho is swapped (ties: the lowest (i, j) in row-major
  order); the swapped-in column takes position i and the swapped-out one position k + j, and R
  is the unpivoted QR of A P (no reordering inside the two blocks).
"""
from __future__ import annotations

import numpy as np

from .linalg import back_substitute


def singular_values(X) -> np.ndarray:
    """Singular values of X in decreasing order (LAPACK through numpy)."""
    return np.linalg.svd(np.asarray(X, dtype=np.float64), compute_uv=False)


def rank_svd(sigma, zeta: float) -> int:
    """Alg. 11 step 3: the number of singular values above zeta * sigma_1 (0 for X = 0)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    if sigma.size == 0 or sigma[0] <= 0:
        return 0
    return int(np.sum(sigma > zeta * sigma[0]))


def r_factor(X, perm) -> np.ndarray:
    """R of the unpivoted QR of X[:, perm] with diag(R) >= 0 (min(m, d) x d)."""
    R = np.linalg.qr(np.asarray(X, dtype=np.float64)[:, np.asarray(perm)], mode="r")
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return R * sgn[:, None]


def srrqr_measures(R: np.ndarray, k: int):
    """rho (k x (d - k)), R11^{-1} R12, gamma (d - k) and 1/omega (k) from R in pivot order."""
    d = R.shape[1]
    R11, R12 = R[:k, :k], R[:k, k:]
    W = back_substitute(R11, np.eye(k))                 # R11^{-1}
    X = W @ R12
    inv_omega = np.sqrt(np.sum(W * W, axis=1))           # ||e_i^T R11^{-1}||
    gamma = np.sqrt(np.sum(R[k:, k:] ** 2, axis=0)) if R.shape[0] > k else np.zeros(d - k)
    rho = np.sqrt(X ** 2 + (gamma[None, :] * inv_omega[:, None]) ** 2)
    return rho, X, gamma, inv_omega


def srrqr(X, k: int, phi: float, perm0, max_swaps: int = 10000):
    """Gu-Eisenstat swaps at fixed k from the column order perm0. Returns (perm, rhos, dets):
    the final order, rho of each swap made, and |det R11| before each swap and at the end."""
    if phi < 1:
        raise ValueError("phi must be >= 1")
    perm = np.asarray(perm0, dtype=np.int64).copy()
    d = perm.size
    dets, rhos = [], []
    while True:
        R = r_factor(X, perm)
        dets.append(float(np.prod(np.abs(np.diag(R)[:k]))))
        if k == 0 or k >= d:
            break
        rho = srrqr_measures(R, k)[0]
        i, j = np.unravel_index(int(np.argmax(rho)), rho.shape)
        if rho[i, j] <= phi:
            break
        if len(rhos) == max_swaps:
            raise RuntimeError("strong RRQR did not settle")
        perm[i], perm[k + j] = perm[k + j], perm[i]
        rhos.append(float(rho[i, j]))
    return perm, rhos, dets
