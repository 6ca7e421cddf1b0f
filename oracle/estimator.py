"""Oracle of the rank-revealing leverage-score estimator (FP64, numpy).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

The estimator is Alg. 10 (LS-HRN-approx): Alg. 4 (CountGaussSRRQR: the
CountGauss sketch of Alg. 3, then a rank-revealing QR of the sketch) selects
the columns K and gives R_11; then steps 4-5 of Alg. 8 run on A_{:,K} with
the orthogonaliser R_11 and a Gaussian JL matrix Omega (the squared row norms of
A (Pi_1 A)^+ Pi_2 of eq. (10): theta~_i = ||e_i^T A_K R_11^{-1} Omega||^2).

Step order (each function cites its step):
 1. hash and sign of every row (CountSketch definition, Sec. 3.4.3);
 2. B = S A, summed in FP64 (Alg. 3, step 3, first product);
 3. A~ = G B with G = N(0,1)/sqrt(m) (Alg. 3 step 3, Sec. 3.4.1 scaling);
 4. pivoted QR of A~, rank r, R_11 (Alg. 4 step 2, xGEQP3-style, Sec. 7);
 5. Omega (r x k) = N(0,1)/sqrt(k), rows indexed by pivot position;
 6. M = R_11^{-1} Omega (Alg. 8 step 4 with the QR orthogonaliser);
 7. theta~_i = sum_q (sum_{p<r} A[i, P_p] M[p, q])^2 (Alg. 8 step 5).

Readings where the paper is silent (also listed in the design notes):
 * G is scaled by 1/sqrt(m) and Omega by 1/sqrt(k) so that theta~ ~ theta;
 * Alg. 10 re-uses the sketch and R_11 of Alg. 4 for Alg. 8 (no second sketch);
 * Omega is indexed by pivot position p (theta~ depends on the pivot order);
 * an all-zero row gets theta~ = 0; a rank-0 input gives theta~ = 0.

Modes: ``sketch_identity`` replaces S and G by identities (s = m = n) and
``omega_identity`` replaces Omega by I_r (k = r); with both, theta~ is the exact
leverage of A_K (Theorem 1, Sec. 2.2, with k = rank(A) gives equality).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import rng
from .linalg import pivoted_qr, back_substitute


def _as_float64(A):
    if sp.issparse(A):
        return A.astype(np.float64).tocsr()
    return np.asarray(A, dtype=np.float64)


def count_sketch(A, s: int, seed: int, block: int = 1 << 18, row0: int = 0) -> np.ndarray:
    """B = S A (s x d), S the CountSketch of rows 0..n-1 (Sec. 3.4.3), FP64 sums.

    With row0 > 0, A is the block of rows row0..row0+n-1 of a larger matrix and the result is
    S_{:,row0:row0+n} A: each row is hashed by its global index (block matrix product)."""
    n, d = A.shape
    B = np.zeros((s, d))
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        b, sign = rng.bucket_and_sign(r1 - r0, s, seed, start=row0 + r0)
        S = sp.csr_matrix((sign, (b, np.arange(r1 - r0))), shape=(s, r1 - r0))
        blk = _as_float64(A[r0:r1])
        prod = S @ blk
        B += prod.toarray() if sp.issparse(prod) else prod
    return B


def gaussian_stage(B: np.ndarray, m: int, seed: int, block: int = 1 << 14) -> np.ndarray:
    """A~ = G B with G (m x s) = N(0,1)/sqrt(m), generated in column blocks."""
    s, d = B.shape
    At = np.zeros((m, d))
    for c0 in range(0, s, block):
        c1 = min(s, c0 + block)
        At += rng.gaussian_sketch_block(m, s, seed, c0, c1) @ B[c0:c1]
    return At


def fwht(X: np.ndarray) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform along axis 0 (length a power of two): butterflies
    (x_i, x_{i+h}) -> (x_i + x_{i+h}, x_i - x_{i+h}) within blocks of 2h, h = 1, 2, 4, ...; the
    result is H X with H_{ij} = (-1)^{popcount(i & j)} (Sylvester order)."""
    X = np.array(X, dtype=np.float64)
    n = X.shape[0]
    assert n & (n - 1) == 0
    tail = X.shape[1:]
    h = 1
    while h < n:
        Y = X.reshape((n // (2 * h), 2, h) + tail)
        a = Y[:, 0].copy()
        Y[:, 0] += Y[:, 1]
        Y[:, 1] = a - Y[:, 1]
        X = Y.reshape((n,) + tail)
        h *= 2
    return X


def srht(B: np.ndarray, t: int, seed: int) -> np.ndarray:
    """C = F B with the SRHT F = sqrt(s/t) P H D of Sec. 3.4.2 (t x s): D the signs of stream 4,
    H the Walsh-Hadamard matrix scaled by 1/sqrt(s), P t uniform row draws (stream 5)."""
    s = B.shape[0]
    X = fwht(rng.srht_signs(s, seed)[:, None] * B)
    return X[rng.srht_rows(t, s, seed)] / np.sqrt(t)


def sketch(A, s: int, m: int, seed: int, srht_t: int = 0, row0: int = 0) -> np.ndarray:
    """CountGauss sketch A~ = G (S A) of Alg. 3 (FP64); with srht_t > 0 the CountSketch is
    followed by an SRHT to t rows (S~ = F S, Sec. 4.1) and G is m x t. With row0 > 0, A is a
    block of rows starting at global row row0 (see count_sketch)."""
    B = count_sketch(A, s, seed, row0=row0)
    if srht_t:
        B = srht(B, srht_t, seed)
    return gaussian_stage(B, m, seed)


def omega_factor(R11: np.ndarray, k: int, seed: int, omega_identity: bool = False) -> np.ndarray:
    """M = R_11^{-1} Omega (r x k), Alg. 8 step 4 with X = R^{-1} Pi_2."""
    r = R11.shape[0]
    Om = np.eye(r) if omega_identity else rng.omega(r, k, seed)
    return back_substitute(R11, Om)


def m_full(M: np.ndarray, perm, d: int) -> np.ndarray:
    """Scatter M (r x k) into a d x k matrix: row perm[p] holds M[p, :], other rows 0."""
    r, k = M.shape
    out = np.zeros((d, k))
    out[np.asarray(perm[:r])] = M
    return out


def final_pass(A, perm, r: int, M: np.ndarray, block: int = 1 << 16) -> np.ndarray:
    """theta~_i = sum_q (sum_{p<r} A[i, P_p] M[p, q])^2 (Alg. 8 step 5), FP64."""
    n = A.shape[0]
    cols = np.asarray(perm[:r], dtype=np.int64)
    theta = np.zeros(n)
    if r == 0:
        return theta
    for r0 in range(0, n, block):
        blk = _as_float64(A[r0:r0 + block])
        AK = blk[:, cols]
        Y = AK @ M
        Y = Y.toarray() if sp.issparse(Y) else np.asarray(Y)
        theta[r0:r0 + block] = np.sum(Y * Y, axis=1)
    return theta


class Estimate:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def estimate(A, s: int, m: int, k: int, tau: float, seed: int, *,
             sketch_identity: bool = False, omega_identity: bool = False,
             forced_perm=None, forced_rank=None, Atilde=None, srht_t: int = 0,
             rank_rule: str = "diag", srrqr_phi: float = 0.0) -> Estimate:
    """Alg. 10 end to end: returns theta (n), rank, perm (d), Atilde, R (r x d), M (r x k).

    ``Atilde`` may be passed in to run steps 4-7 on a given sketch. ``rank_rule="svd"`` takes
    the rank from the singular values of the sketch (Alg. 11 step 3, Sec. 7.2) and the columns
    from its pivoted QR run to the end; ``srrqr_phi >= 1`` then improves the selected columns by
    strong-RRQR swaps at that rank (oracle/rank.py).
    """
    n, d = A.shape
    if Atilde is None:
        if sketch_identity:
            Atilde = _as_float64(A)
            Atilde = Atilde.toarray() if sp.issparse(Atilde) else np.array(Atilde)
        else:
            Atilde = sketch(A, s, m, seed, srht_t)
    if forced_perm is None and (rank_rule != "diag" or srrqr_phi):
        from . import rank as rank_mod
        if rank_rule == "svd":
            forced_perm = pivoted_qr(Atilde, 0.0).perm
            forced_rank = rank_mod.rank_svd(rank_mod.singular_values(Atilde), tau)
        elif rank_rule == "diag":
            qr0 = pivoted_qr(Atilde, tau)
            forced_perm, forced_rank = qr0.perm, qr0.rank
        else:
            raise ValueError(f"unknown rank rule {rank_rule}")
        if srrqr_phi:
            forced_perm = rank_mod.srrqr(Atilde, forced_rank, srrqr_phi, forced_perm)[0]
    qr = pivoted_qr(Atilde, tau, forced_perm=forced_perm, forced_rank=forced_rank)
    r = qr.rank
    if r == 0:
        return Estimate(theta=np.zeros(n), rank=0, perm=qr.perm, Atilde=Atilde,
                        R=qr.R, M=np.zeros((0, k)), qr=qr)
    R11 = qr.R[:, :r]
    M = omega_factor(R11, k, seed, omega_identity)
    theta = final_pass(A, qr.perm, r, M)
    return Estimate(theta=theta, rank=r, perm=qr.perm, Atilde=Atilde, R=qr.R, M=M, qr=qr)
