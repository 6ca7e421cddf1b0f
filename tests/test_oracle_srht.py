"""Pins for the oracle's SRHT (Sec. 3.4.2) and the CountSketch + SRHT + Gaussian sketch (Sec. 4.1).

The Walsh-Hadamard transform against scipy's Hadamard matrix and its involution, the sign and
row draws against their distributions, the subspace-embedding bounds of the SRHT theorem the
paper quotes (Tropp 2011, Thm. 3.1) and exact leverage recovered by Alg. 7 with the SRHT sketch.
"""
import numpy as np
import scipy.linalg

import workloads as W
from oracle import estimator as E, exact as X, rng


def test_fwht_equals_hadamard_matrix():
    Y = np.random.default_rng(0).standard_normal((64, 5))
    np.testing.assert_allclose(E.fwht(Y), scipy.linalg.hadamard(64) @ Y, rtol=0, atol=1e-12)


def test_fwht_twice_is_n_times_identity():
    Y = np.random.default_rng(1).standard_normal((1024, 3))
    np.testing.assert_allclose(E.fwht(E.fwht(Y)), 1024 * Y, rtol=0, atol=1e-9)


def test_signs_and_rows_are_balanced():
    sg = rng.srht_signs(1 << 16, seed=3)
    assert abs(sg.mean()) < 0.02
    rows = rng.srht_rows(64000, 64, seed=3)
    assert rows.min() == 0 and rows.max() == 63
    counts = np.bincount(rows, minlength=64)
    chi2 = float(np.sum((counts - 1000.0) ** 2 / 1000.0))
    assert chi2 < 120.0                          # 63 degrees of freedom; p ~ 1e-5 at 120


def test_srht_subspace_embedding_bounds():
    """Thm. 3.1 as quoted: t >= 4 (sqrt(d) + sqrt(ln(s d)))^2 ln d gives singular values of F U
    in [sqrt(1/6), sqrt(13/6)] (probability >= 1 - 3/d; checked on three seeds)."""
    s, d = 4096, 10
    t = int(np.ceil(4 * (np.sqrt(d) + np.sqrt(np.log(s * d))) ** 2 * np.log(d)))
    U, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((s, d)))
    for seed in range(3):
        sv = np.linalg.svd(E.srht(U, t, seed), compute_uv=False)
        assert sv.min() >= np.sqrt(1 / 6) and sv.max() <= np.sqrt(13 / 6)


def test_srht_is_unbiased_on_average():
    """E[F^T F] = I: the average of ||F x||^2 over seeds approaches ||x||^2."""
    x = np.random.default_rng(2).standard_normal((256, 1))
    vals = [float(np.sum(E.srht(x, 32, seed) ** 2)) for seed in range(400)]
    assert abs(np.mean(vals) / float(np.sum(x * x)) - 1.0) < 0.05


def test_ls_hrn_exact_with_srht_sketch_is_exact_at_full_rank():
    A = W.dense_heavy_rows(600, 10, seed=6).astype(np.float64)
    th, k, _ = X.ls_hrn_exact(A, s=512, m=40, tau=1e-10, seed=4, srht_t=200)
    assert k == 10
    H = A @ np.linalg.pinv(A.T @ A) @ A.T
    np.testing.assert_allclose(th, np.diag(H), rtol=0, atol=1e-10)


def test_srht_rows_are_the_top_bits_for_a_power_of_two_s():
    """Multiply-shift of the high word: for s = 2^q a row is the top q bits of the high word of
    stream 5 (a modulo would take the low ones)."""
    s, t, seed = 1 << 10, 300, 4
    x = rng.splitmix64(rng.stream_key(seed, rng.STREAM_SRHT_ROWS), np.arange(t))
    top = (x >> np.uint64(54)).astype(np.int64)
    assert np.array_equal(rng.srht_rows(t, s, seed), top)


def test_srht_signs_are_bit_0_of_stream_4():
    """D of the SRHT: +1 where bit 0 of the stream-4 word is 0, else -1 (the published definition)."""
    x = rng.splitmix64(rng.stream_key(5, rng.STREAM_SRHT_SIGN), np.arange(256))
    want = np.where((x & np.uint64(1)) == 0, 1.0, -1.0)
    assert np.array_equal(rng.srht_signs(256, 5), want)
    assert np.array_equal(rng.srht_signs(256, 5), rng.srht_signs(300, 5)[:256])


def test_srht_equals_its_explicit_matrix_product():
    """F = sqrt(s/t) P H D (Sec. 3.4.2) built as explicit matrices (scipy's Sylvester Hadamard
    scaled by 1/sqrt(s), the stream-4 signs on the diagonal of D, the stream-5 rows in P): F B
    equals the oracle's srht(B); D acts before H."""
    s, t, seed = 64, 20, 3
    B = np.random.default_rng(0).standard_normal((s, 5))
    H = scipy.linalg.hadamard(s) / np.sqrt(s)
    D = np.diag(rng.srht_signs(s, seed))
    P = np.zeros((t, s))
    P[np.arange(t), rng.srht_rows(t, s, seed)] = 1.0
    F = np.sqrt(s / t) * P @ H @ D
    np.testing.assert_allclose(E.srht(B, t, seed), F @ B, atol=1e-12)
