"""The seeded input generators (workloads/) produce the matrices their recipes state; no GPU."""
import numpy as np
import scipy.sparse as sp

import workloads as W


def _dense(C):
    return sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=C.shape)


def test_dense_lowrank_skewed_has_the_stated_rank_and_is_block_invariant():
    A = W.dense_lowrank_skewed(3000, 40, 25, seed=9)
    assert A.shape == (3000, 40) and A.dtype == np.float32
    s = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    assert s[24] / s[0] > 1e-3 and s[25] / s[0] < 1e-5        # rank 25 up to the FP32 rounding
    assert np.array_equal(W.dense_lowrank_skewed(3000, 40, 25, seed=9, block=700), A)
    assert np.array_equal(W.dense_lowrank_skewed(3000, 40, 25, seed=9), A)
    assert not np.array_equal(W.dense_lowrank_skewed(3000, 40, 25, seed=10), A)


def test_csr_uniform_rows_and_heavy_fraction():
    n, d = 40000, 1024
    C = W.csr_uniform(n, d, seed=2)
    counts = np.diff(C.row_ptr)
    assert set(np.unique(counts).tolist()) == {8, 256}
    frac = np.mean(counts == 256)
    assert abs(frac - 0.01) < 5 * np.sqrt(0.01 * 0.99 / n)
    assert C.col.min() >= 0 and C.col.max() < d and C.col.dtype == np.int32
    for i in np.random.default_rng(0).integers(0, n, 500):
        row = C.col[C.row_ptr[i]:C.row_ptr[i + 1]]
        assert np.all(np.diff(row) > 0)                        # distinct and sorted
    assert abs(C.val.astype(np.float64).std() - 1) < 0.02


def test_csr_dup_columns_pairs_are_exact_doubles():
    n, d, pairs = 30000, 64, 10
    C = W.csr_dup_columns(n, d, nnz_per_row=12, pairs=pairs, seed=5)
    A = _dense(C).toarray()
    half = d // 2
    for j in range(pairs):
        assert np.array_equal(A[:, j + half], 2.0 * A[:, j])   # exact in FP32 (a doubling)
        assert np.count_nonzero(A[:, j]) > 0
    assert np.linalg.matrix_rank(A) == d - pairs
    counts = np.diff(C.row_ptr)
    assert counts.min() >= 12 and np.all((counts - 12) == np.sum(A[:, :pairs] != 0, axis=1))


def test_fixed_svd_has_the_prescribed_singular_values():
    sig = np.concatenate([np.ones(15), np.full(15, 1e-6), np.full(30, 1e-7)])
    A = W.fixed_svd(5000, 60, sig, seed=7)
    np.testing.assert_allclose(np.linalg.svd(A, compute_uv=False), sig, rtol=1e-7, atol=1e-15)


def test_dense_heavy_rows_scale_a_bernoulli_subset():
    A = W.dense_heavy_rows(20000, 64, heavy_frac=0.05, factor=100.0, seed=3)
    norms = np.linalg.norm(A.astype(np.float64), axis=1)
    heavy = norms > 10 * np.sqrt(64)
    assert abs(heavy.mean() - 0.05) < 5 * np.sqrt(0.05 * 0.95 / 20000)
    assert np.all((norms[heavy] / 100 > 4) & (norms[heavy] / 100 < 12))
