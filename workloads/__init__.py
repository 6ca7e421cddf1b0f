"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds input matrices and weights. It holds none of the
estimator's arithmetic (no hash, no sketch, no Gaussian stream of the method),
so both the CPU oracle and the CUDA path can read the same bytes from it.

Every generator uses ``numpy.random.default_rng(seed)`` (PCG64), computes in
FP64 and rounds to the requested storage type at the end.

Workload shapes (the paper's own datasets, timg80 and kl02 of Sec. 7.1, are
not available; these stand in for them with the same roles):

* ``dense_gaussian``      -- small full-rank dense matrix (correctness case).
* ``dense_lowrank_skewed``-- tall dense A = diag(e^{2 z}) U V^T, exact rank,
                             lognormal(0, 2) row scaling for skewed leverage.
* ``csr_uniform``         -- tall CSR matrix, a few uniform random columns per
                             row plus a small fraction of heavy rows.
* ``dense_heavy_rows``    -- N(0,1) dense matrix with a fraction of rows x100
                             (the backward-pass workload) and U(0,1) weights.
* ``csr_dup_columns``     -- tall CSR matrix shaped like timg80 (Sec. 7.1,
                             Table 6: 79,302,017 x 1,024) with column pairs
                             made exactly dependent (column j+d/2 = 2 x col j).
* ``fixed_svd``           -- dense matrix with a prescribed singular-value
                             profile and seeded Haar-orthogonal factors (the
                             fixed_svd_* matrices of Sec. 7.1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "CSR",
    "dense_gaussian",
    "dense_lowrank_skewed",
    "csr_uniform",
    "dense_heavy_rows",
    "csr_dup_columns",
    "fixed_svd",
    "uniform_weights",
    "CONFIGS",
]


class CSR:
    """Plain CSR container: int64 row_ptr (n+1), int32 col (nnz), val (nnz)."""

    def __init__(self, row_ptr, col, val, shape):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val)
        self.shape = (int(shape[0]), int(shape[1]))

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def astype(self, dtype) -> "CSR":
        return CSR(self.row_ptr, self.col, self.val.astype(dtype), self.shape)

    def to_dense(self) -> np.ndarray:
        n, d = self.shape
        out = np.zeros((n, d), dtype=np.float64)
        rows = np.repeat(np.arange(n), np.diff(self.row_ptr))
        np.add.at(out, (rows, self.col), self.val.astype(np.float64))
        return out

    def row_slice(self, r0: int, r1: int) -> "CSR":
        a, b = int(self.row_ptr[r0]), int(self.row_ptr[r1])
        return CSR(self.row_ptr[r0:r1 + 1] - a, self.col[a:b], self.val[a:b],
                   (r1 - r0, self.shape[1]))


def dense_gaussian(n: int, d: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """A with i.i.d. N(0,1) entries, row-major."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((n, d)).astype(dtype))


def dense_lowrank_skewed(n: int, d: int, rank: int, seed: int = 1,
                         log_sigma: float = 2.0, dtype=np.float32,
                         block: int = 1 << 18) -> np.ndarray:
    """A = diag(exp(log_sigma * z)) U V^T with U (n x rank), V (d x rank), z ~ N(0,1).

    Formed in FP64 row block by row block and rounded to ``dtype``; the exact
    rank of the FP64 product is ``rank``.
    """
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((d, rank))
    z = rng.standard_normal(n)
    out = np.empty((n, d), dtype=dtype)
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        U = rng.standard_normal((r1 - r0, rank))
        blk = (U @ V.T) * np.exp(log_sigma * z[r0:r1])[:, None]
        out[r0:r1] = blk.astype(dtype)
    return out


def _distinct_sorted_columns(rng, rows: int, per_row: int, d: int) -> np.ndarray:
    """rows x per_row distinct uniform column indices in [0, d), sorted per row."""
    if per_row * 4 >= d:
        keys = rng.random((rows, d))
        cols = np.argpartition(keys, per_row - 1, axis=1)[:, :per_row]
        return np.sort(cols, axis=1).astype(np.int32)
    cols = np.sort(rng.integers(0, d, size=(rows, per_row)), axis=1)
    while True:
        bad = np.nonzero((np.diff(cols, axis=1) == 0).any(axis=1))[0]
        if bad.size == 0:
            break
        cols[bad] = np.sort(rng.integers(0, d, size=(bad.size, per_row)), axis=1)
    return cols.astype(np.int32)


def csr_uniform(n: int, d: int, nnz_per_row: int = 8, heavy_frac: float = 0.01,
                heavy_nnz: int = 256, seed: int = 2, dtype=np.float32) -> CSR:
    """CSR with ``nnz_per_row`` distinct uniform columns per row, N(0,1) values.

    A ``heavy_frac`` fraction of rows (chosen by a Bernoulli draw) has
    ``heavy_nnz`` columns instead. Columns are sorted within each row.
    """
    rng = np.random.default_rng(seed)
    heavy = rng.random(n) < heavy_frac
    counts = np.where(heavy, heavy_nnz, nnz_per_row).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = np.empty(int(row_ptr[-1]), dtype=np.int32)
    light_rows = np.nonzero(~heavy)[0]
    heavy_rows = np.nonzero(heavy)[0]
    lc = _distinct_sorted_columns(rng, light_rows.size, nnz_per_row, d)
    idx = row_ptr[light_rows][:, None] + np.arange(nnz_per_row)[None, :]
    col[idx.ravel()] = lc.ravel()
    for h0 in range(0, heavy_rows.size, 4096):
        hr = heavy_rows[h0:h0 + 4096]
        hc = _distinct_sorted_columns(rng, hr.size, heavy_nnz, d)
        idx = row_ptr[hr][:, None] + np.arange(heavy_nnz)[None, :]
        col[idx.ravel()] = hc.ravel()
    val = rng.standard_normal(col.size).astype(dtype)
    return CSR(row_ptr, col, val, (n, d))


def dense_heavy_rows(n: int, d: int, heavy_frac: float = 0.05, factor: float = 100.0,
                     seed: int = 3, dtype=np.float32) -> np.ndarray:
    """N(0,1) entries; a Bernoulli(heavy_frac) subset of rows multiplied by ``factor``."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, d))
    heavy = rng.random(n) < heavy_frac
    A[heavy] *= factor
    return np.ascontiguousarray(A.astype(dtype))


def uniform_weights(n: int, seed: int = 4, dtype=np.float32) -> np.ndarray:
    """w_i ~ U(0, 1)."""
    return np.random.default_rng(seed).random(n).astype(dtype)


def csr_dup_columns(n: int, d: int, nnz_per_row: int = 12, pairs: int = 10,
                    seed: int = 5, dtype=np.float32, block: int = 1 << 20) -> CSR:
    """CSR shaped like timg80 with ``pairs`` exactly dependent column pairs.

    Each row draws ``nnz_per_row`` distinct uniform columns from the columns
    that are not dependent copies; whenever column j < pairs is present, the
    entry (j + d/2, 2 * value) is added, so column j + d/2 equals exactly twice
    column j and rank(A) = d - pairs (with high probability).
    """
    rng = np.random.default_rng(seed)
    half = d // 2
    dep = np.arange(pairs) + half                       # dependent copies
    free = np.setdiff1d(np.arange(d), dep).astype(np.int32)
    rows_cols, rows_vals, counts = [], [], np.empty(n, dtype=np.int64)
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        nb = r1 - r0
        c = free[_distinct_sorted_columns(rng, nb, nnz_per_row, free.size)]
        v = rng.standard_normal((nb, nnz_per_row))
        pmask = c < pairs                                # a row can hold several pair columns
        extra = pmask.sum(axis=1)
        counts[r0:r1] = nnz_per_row + extra
        if extra.any():
            cc = np.concatenate([c, np.where(pmask, c + half, d)], axis=1)
            vv = np.concatenate([v, np.where(pmask, 2.0 * v, 0.0)], axis=1)
            order = np.argsort(cc, axis=1, kind="stable")
            cc = np.take_along_axis(cc, order, axis=1)
            vv = np.take_along_axis(vv, order, axis=1)
            keep = cc < d
            rows_cols.append(cc[keep].astype(np.int32))
            rows_vals.append(vv[keep])
        else:
            rows_cols.append(c.ravel().astype(np.int32))
            rows_vals.append(v.ravel())
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = np.concatenate(rows_cols)
    val = np.concatenate(rows_vals).astype(dtype)
    return CSR(row_ptr, col, val, (n, d))


def _haar_orthogonal(rng, n: int, k: int) -> np.ndarray:
    """n x k matrix with orthonormal columns, Haar distributed (QR of a Gaussian, sign-fixed)."""
    Z = rng.standard_normal((n, k))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def fixed_svd(n: int, d: int, sigmas, seed: int = 7, dtype=np.float64) -> np.ndarray:
    """A = U diag(sigmas) V^T with seeded Haar-orthogonal U (n x d) and V (d x d)."""
    rng = np.random.default_rng(seed)
    sig = np.asarray(sigmas, dtype=np.float64)
    assert sig.size == d
    U = _haar_orthogonal(rng, n, d)
    V = _haar_orthogonal(rng, d, d)
    return np.ascontiguousarray(((U * sig[None, :]) @ V.T).astype(dtype))


# Workload table: sizes and method parameters of the five workloads the
# estimator is measured on. ``tau`` is the rank-rule threshold |R_jj| > tau |R_00|.
CONFIGS = {
    "dense_2000x20_f64": dict(kind="dense", n=2000, d=20, s=1600, m=80, k=64,
                              tau=1e-10, seed=0, data_seed=0),
    "dense_1e6x256_rank200": dict(kind="dense", n=1_000_000, d=256, rank=200, s=65536,
                                  m=1024, k=256, tau=1e-4, seed=11, data_seed=1),
    "csr_8e6x1024": dict(kind="csr", n=8_000_000, d=1024, s=262144, m=4096, k=256,
                         tau=1e-5, seed=12, data_seed=2),
    "dense_2e5x64_backward": dict(kind="dense", n=200_000, d=64, s=16384, m=256, k=128,
                                  tau=1e-5, seed=13, data_seed=3, weight_seed=4),
    "csr_8e7x1024_rank1014": dict(kind="csr", n=80_000_000, d=1024, s=262144, m=4096,
                                  k=256, tau=1e-5, seed=15, data_seed=5),
}
