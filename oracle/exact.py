"""Oracle exact leverage scores (FP64, numpy).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

Definition (Sec. 1, eq. (1) and the paragraph after it): theta_i = diag(H)_i
with H = A (A^T A)^+ A^T, equivalently the squared row norms of any matrix
whose columns are an orthonormal basis of range(A).

Two routes:
* ``exact_leverage_qr``: column-pivoted Householder QR of A (the rank rule of
  Sec. 7.2 on diag(R)); theta_i = ||Q[i, :rank]||^2.
* ``exact_leverage_gram``: Alg. 5 (Gram matrix A^T A formed as a sum of row
  outer products, Lemma 8, Sec. 5.1; symmetric eigendecomposition; keep eigenvalues
  lambda_j > tau^2 lambda_max; theta_i = ||A_i V_k Lambda_k^{-1/2}||^2).

And Alg. 7 (LS-HRN-exact), ``ls_hrn_exact``: the columns K and the rank k come
from the pivoted QR of the CountGauss sketch (Alg. 4), then the exact scores of
A_K by its Gram matrix (steps 4-6).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .linalg import pivoted_qr
from .estimator import sketch


def exact_leverage_qr(A: np.ndarray, tau: float):
    """(theta, rank) from the pivoted QR of dense A (n x d), FP64."""
    A = np.asarray(A, dtype=np.float64)
    qr = pivoted_qr(A, tau)
    if qr.rank == 0:
        return np.zeros(A.shape[0]), 0
    Q = qr.q_thin(qr.rank)
    return np.sum(Q * Q, axis=1), qr.rank


def gram(A, block: int = 1 << 16) -> np.ndarray:
    """A^T A accumulated over row blocks (Lemma 8, Sec. 5.1: sum of row outer products)."""
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


def ls_hrn_exact(A, s: int, m: int, tau: float, seed: int, *, sketch_identity: bool = False,
                 block: int = 1 << 16, srht_t: int = 0):
    """Alg. 7 (LS-HRN-exact), FP64. Returns (theta, rank, perm).

    Steps 1-3: K and k from the column-pivoted QR of the sketch A~ = G S A (Alg. 3 and 4, the
    GEQP3-style pivoting and rank rule of Sec. 7; A~ = A when ``sketch_identity``); A_K = A P_k.
    Step 4: B = A_K^T A_K as a sum of row outer products (Lemma 8, Sec. 5.1).
    Step 5: B = V Sigma^2 V^T (B is symmetric positive definite when the k columns are linearly
    independent, so its SVD is its eigendecomposition).
    Step 6: theta_i = ||e_i^T A_K V Sigma^{-1}||^2.
    """
    n, d = A.shape
    if sketch_identity:
        At = A.toarray() if sp.issparse(A) else np.array(A, dtype=np.float64)
        At = At.astype(np.float64)
    else:
        At = sketch(A, s, m, seed, srht_t)
    qr = pivoted_qr(At, tau)
    k = qr.rank
    if k == 0:
        return np.zeros(n), 0, qr.perm
    K = np.asarray(qr.perm[:k])
    A_K = A.tocsc()[:, K].tocsr() if sp.issparse(A) else np.asarray(A, dtype=np.float64)[:, K]
    B = gram(A_K, block)
    lam, V = np.linalg.eigh(B)
    X = V / np.sqrt(lam)[None, :]
    theta = np.empty(n)
    for r0 in range(0, n, block):
        blk = A_K[r0:r0 + block]
        Y = (blk @ X) if sp.issparse(blk) else np.asarray(blk, dtype=np.float64) @ X
        theta[r0:r0 + block] = np.sum(np.asarray(Y) ** 2, axis=1)
    return theta, k, qr.perm
