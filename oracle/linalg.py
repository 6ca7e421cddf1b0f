"""Oracle column-pivoted Householder QR (FP64, numpy).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

Follows the classical pivoted QR of Businger and Golub that the paper's
implementation uses through LAPACK xGEQP3 (Sec. 7, first paragraph, and
Sec. 7.2), with these readings where the paper is silent:

* pivot rule: at step j the remaining column with the largest trailing norm
  ||W[j:, c]|| is brought to position j; trailing norms are recomputed from
  scratch at every step (no norm downdating); exact ties go to the lowest
  original column index;
* rank rule (Sec. 7.2: the rank is read off the diagonal of R by comparing
  |R_kk| with c |R_11|): r is the number of leading steps with
  |R_jj| > tau |R_00|; the factorisation stops at the first step that fails;
* sign rule: diag(R) >= 0 (rows of R and columns of Q are flipped together).

Because of the exact norm recompute, |R_jj| equals the largest trailing norm
at step j, so the rank test is made before the reflector of step j is built.
"""
from __future__ import annotations

import numpy as np


class PivotedQR:
    """Result of ``pivoted_qr``: perm (d), rank r, R (r x d, permuted columns), reflectors."""

    def __init__(self, perm, rank, R, V, betas, m):
        self.perm = perm
        self.rank = rank
        self.R = R
        self._V = V
        self._betas = betas
        self._m = m

    def q_thin(self, cols: int | None = None) -> np.ndarray:
        """First ``cols`` columns of Q (m x cols), sign-normalised like R."""
        cols = self.rank if cols is None else cols
        Q = np.zeros((self._m, cols))
        Q[np.arange(cols), np.arange(cols)] = 1.0
        for j in range(len(self._V) - 1, -1, -1):
            v, beta = self._V[j], self._betas[j]
            if beta == 0.0:
                continue
            Q[j:, :] -= np.outer(v, beta * (v @ Q[j:, :]))
        return Q * self._signs[None, :cols]


def pivoted_qr(X: np.ndarray, tau: float, max_steps: int | None = None,
               forced_perm=None, forced_rank: int | None = None) -> PivotedQR:
    """Column-pivoted Householder QR of X (m x d) with exact norm recompute.

    With ``forced_perm``/``forced_rank`` the pivot order and rank are taken as
    given (no pivot search, no rank test): this is the QR of X[:, perm[:r]].
    """
    W = np.array(X, dtype=np.float64, copy=True)
    m, d = W.shape
    steps = min(m, d) if max_steps is None else min(m, d, max_steps)
    perm = np.arange(d)
    if forced_perm is not None:
        perm = np.asarray(forced_perm, dtype=np.int64).copy()
        W = W[:, perm]
        steps = min(steps, int(forced_rank))
    R = np.zeros((steps, d))
    V, betas, signs = [], [], []
    r00 = None
    rank = 0
    for j in range(steps):
        if forced_perm is None:
            trailing = np.sqrt(np.sum(W[j:, j:] ** 2, axis=0))
            best = trailing.max()
            ties = np.nonzero(trailing == best)[0] + j
            p = ties[np.argmin(perm[ties])]
            if j == 0:
                r00 = best
            if best == 0.0 or best <= tau * r00:
                break
            if p != j:
                W[:, [j, p]] = W[:, [p, j]]
                R[:j, [j, p]] = R[:j, [p, j]]
                perm[[j, p]] = perm[[p, j]]
        x = W[j:, j].copy()
        nx = np.sqrt(x @ x)
        alpha = -nx if x[0] >= 0 else nx          # reflect x onto alpha e1
        v = x
        v[0] -= alpha
        vv = v @ v
        beta = 2.0 / vv if vv > 0 else 0.0
        if beta != 0.0:
            W[j:, j:] -= np.outer(v, beta * (v @ W[j:, j:]))
        sgn = 1.0 if W[j, j] >= 0 else -1.0
        R[j, :] = 0.0
        R[j, j:] = sgn * W[j, j:]
        V.append(v)
        betas.append(beta)
        signs.append(sgn)
        rank = j + 1
    res = PivotedQR(perm, rank, R[:rank].copy(), V[:rank], betas[:rank], m)
    res._signs = np.asarray(signs[:rank] + [1.0] * max(0, m - rank))
    return res


def back_substitute(R11: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve R11 X = B for upper-triangular R11 by back-substitution (FP64)."""
    r = R11.shape[0]
    X = np.zeros((r, B.shape[1]))
    for p in range(r - 1, -1, -1):
        X[p] = (B[p] - R11[p, p + 1:] @ X[p + 1:]) / R11[p, p]
    return X
