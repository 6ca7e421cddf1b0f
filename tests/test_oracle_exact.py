"""Pins for the oracle's exact leverage scores and pivoted QR (no GPU)."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import exact, linalg


def brute_force_leverage(A):
    """diag(A (A^T A)^+ A^T) with the pseudo-inverse taken by numpy's SVD (Sec. 1, eq. (1))."""
    H = A @ np.linalg.pinv(A.T @ A) @ A.T
    return np.diag(H)


@pytest.mark.parametrize("n,d,seed", [(64, 8, 0), (40, 5, 1), (9, 9, 2)])
def test_qr_route_equals_brute_force(n, d, seed):
    A = W.dense_gaussian(n, d, seed)
    th, r = exact.exact_leverage_qr(A, 1e-12)
    assert r == d
    np.testing.assert_allclose(th, brute_force_leverage(A), atol=1e-12)


def test_gram_route_equals_qr_route():
    A = W.dense_gaussian(2000, 20, 0)
    t1, r1 = exact.exact_leverage_qr(A, 1e-10)
    t2, r2 = exact.exact_leverage_gram(A, 1e-10)
    assert r1 == r2 == 20
    np.testing.assert_allclose(t1, t2, atol=1e-12)


def test_sum_is_rank_and_bounds_rank_deficient():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((300, 5)) @ rng.standard_normal((5, 12))   # rank 5
    th, r = exact.exact_leverage_qr(A, 1e-10)
    assert r == 5
    assert th.sum() == pytest.approx(5.0, abs=1e-10)
    assert th.min() >= -1e-14 and th.max() <= 1 + 1e-12
    np.testing.assert_allclose(th, brute_force_leverage(A), atol=1e-9)


def test_row_alone_in_its_direction_has_leverage_one():
    A = W.dense_gaussian(200, 6, 5)
    e = np.zeros((200, 1))
    e[17] = 3.0
    th, r = exact.exact_leverage_qr(np.hstack([A, e]), 1e-12)
    assert r == 7
    assert th[17] == pytest.approx(1.0, abs=1e-12)


def test_invariance_under_column_transform_and_row_permutation():
    A = W.dense_gaussian(500, 7, 6)
    T = np.random.default_rng(7).standard_normal((7, 7))
    th, _ = exact.exact_leverage_qr(A, 1e-12)
    th_T, _ = exact.exact_leverage_qr(A @ T, 1e-12)
    np.testing.assert_allclose(th, th_T, atol=1e-10)
    p = np.random.default_rng(8).permutation(500)
    th_p, _ = exact.exact_leverage_qr(A[p], 1e-12)
    np.testing.assert_allclose(th_p, th[p], atol=1e-12)


def test_duplicate_rows_split_leverage():
    A = W.dense_gaussian(100, 4, 9)
    th, _ = exact.exact_leverage_qr(A, 1e-12)
    A2 = np.vstack([A, A[3:4]])
    th2, _ = exact.exact_leverage_qr(A2, 1e-12)
    # duplicating row 3: both copies get theta_3 / (1 + theta_3)
    want = th[3] / (1 + th[3])
    assert th2[3] == pytest.approx(want, abs=1e-12)
    assert th2[100] == pytest.approx(want, abs=1e-12)


def test_pivoted_qr_properties():
    A = W.dense_gaussian(80, 12, 10) * np.logspace(0, -3, 12)[None, :]
    q = linalg.pivoted_qr(A, 0.0)
    R = q.R
    Q = q.q_thin(12)
    np.testing.assert_allclose(Q @ R, A[:, q.perm], atol=1e-13)
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-13)
    assert np.all(np.diag(R) >= 0)
    # pivoting: |R_jj| dominates the trailing part of every later column
    for j in range(12):
        for c in range(j, 12):
            assert R[j, j] >= np.linalg.norm(R[j:c + 1, c]) * (1 - 1e-12)
    # R agrees with numpy's QR of the permuted matrix up to row signs
    R_np = np.linalg.qr(A[:, q.perm], mode="r")
    np.testing.assert_allclose(np.abs(R_np), np.abs(R), atol=1e-12)


def test_pivot_tie_goes_to_lowest_original_index():
    A = np.zeros((10, 4))
    A[:, 1] = np.arange(10.0)
    A[:, 3] = np.arange(10.0)
    q = linalg.pivoted_qr(A, 1e-10)
    assert q.perm[0] == 1 and q.rank == 1


def test_rank_zero_matrix():
    th, r = exact.exact_leverage_qr(np.zeros((10, 3)), 1e-10)
    assert r == 0 and np.all(th == 0)


def _paper_rank_rows(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "paper_ranks.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                rows.append(ln.split())
    return rows


def _profile(spec):
    parts = []
    for item in spec.split(","):
        v, c = item.split(":")
        parts.append(np.full(int(c), float(v)))
    return np.concatenate(parts)


@pytest.mark.slow
def test_paper_stated_ranks(golden_dir):
    """Ranks the paper states for fixed_svd_2.5e4 and fixed_svd_1e7 (Sec. 7.2, 7.4)."""
    from oracle import estimator
    for name, n, d, prof, thr, rule, want in _paper_rank_rows(golden_dir):
        n, d, thr = int(n), int(d), float(thr)
        A = W.fixed_svd(n, d, _profile(prof), seed=7)
        if rule == "svd":
            sv = np.linalg.svd(A, compute_uv=False)
            got = int(np.sum(sv > thr * sv[0]))
            assert got == int(want), name
            assert exact.exact_leverage_gram(A, thr)[1] == int(want), name
        elif rule == "qr":
            got = linalg.pivoted_qr(A, thr).rank
            assert want == "not30" and got != 30, name
        elif rule == "qr_sketch":
            # Alg. 4 on the CountGauss sketch with m = 2d, r = 5(d^2 + d) (Sec. 7.2)
            e = estimator.estimate(A, 5 * (d * d + d), 2 * d, d, thr, seed=3)
            assert e.rank == int(want), name


def test_gram_blocks_sum_to_the_gram_matrix():
    """Lemma 8 (Sec. 5.1): A^T A as the sum over row blocks of their outer products, dense and
    CSR, with blocks far smaller than n (the sum of all blocks, not the last one)."""
    import scipy.sparse as sp
    A = np.random.default_rng(3).standard_normal((103, 7))
    np.testing.assert_allclose(exact.gram(A, block=16), A.T @ A, rtol=1e-13, atol=1e-12)
    C = sp.random(103, 7, density=0.3, random_state=4, format="csr")
    np.testing.assert_allclose(exact.gram(C, block=10), (C.T @ C).toarray(), rtol=1e-13, atol=1e-12)
