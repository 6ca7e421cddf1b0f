"""Oracle exact leverage scores (FP64, numpy).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

Definition (Sec. 1, eq. (1) and the paragraph after it): theta_i = diag(H)_i
with H = A (A^T A)^+ A^T, equivalently the squared row norms of any matrix
whose columns are an orthonormal basis of range(A).

Two routes:
* ``exact_leverage_qr``: column-pivoted Householder QR of A (the rank rule of
  Sec. 6.2 on diag(R)); theta_i = ||Q[i, :rank]||^2.
* ``exact_leverage_gram``: Alg. 5 (Gram matrix A^T A formed as a sum of row
  outer products, Lemma 3; symmetric eigendecomposition; keep eigenvalues
  lambda_j > tau^2 lambda_max; theta_i = ||A_i V_k Lambda_k^{-1/2}||^2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .linalg import pivoted_qr


def exact_leverage_qr(A: np.ndarray, tau: float):
    """(theta, rank) from the pivoted QR of dense A (n x d), FP64."""
    A = np.asarray(A, dtype=np.float64)
    qr = pivoted_qr(A, tau)
    if qr.rank == 0:
        return np.zeros(A.shape[0]), 0
    Q = qr.q_thin(qr.rank)
    return np.sum(Q * Q, axis=1), qr.rank


def gram(A, block: int = 1 << 16) -> np.ndarray:
    """A^T A accumulated over row blocks (Lemma 3: sum of row outer products)."""
    d = A.shape[1]
    Gm = np.zeros((d, d))
    for r0 in range(0, A.shape[0], block):
        blk = A[r0:r0 + block]
        if sp.issparse(blk):
            blk = blk.astype(np.float64)
            Gm += (blk.T @ blk).toarray()
        else:
            blk = np.asarray(blk, dtype=np.float64)
            Gm += blk.T @ blk
    return Gm


def exact_leverage_gram(A, tau: float, block: int = 1 << 16):
    """(theta, rank) by Alg. 5 for dense or scipy-sparse A; rank rule sigma_j > tau sigma_1."""
    Gm = gram(A, block)
    lam, V = np.linalg.eigh(Gm)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    if lam[0] <= 0:
        return np.zeros(A.shape[0]), 0
    keep = lam > (tau * tau) * lam[0]
    k = int(np.sum(keep))
    X = V[:, :k] / np.sqrt(lam[:k])[None, :]
    theta = np.empty(A.shape[0])
    for r0 in range(0, A.shape[0], block):
        blk = A[r0:r0 + block]
        Y = (blk @ X) if sp.issparse(blk) else np.asarray(blk, dtype=np.float64) @ X
        theta[r0:r0 + block] = np.sum(np.asarray(Y) ** 2, axis=1)
    return theta, k
