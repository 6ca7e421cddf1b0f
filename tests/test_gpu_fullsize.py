"""Full-size parity: the workload sizes, in the launch configuration bench.py times.

At these sizes the oracle recomputes what it can one entry at a time, on the GPU's
own intermediates:
* sketch: sampled entries A~[j, c] = G[j, :] . (S A)[:, c] (one G row, one sketch column);
* QR: pivots form a permutation, diag(R) > 0, the Gram identity
  (A~ P)^T (A~ P) = R^T R on sampled entries of the leading r x r block, the rank;
* final pass: theta~ of sampled rows from the GPU's Mfull, in FP64.
The end-to-end comparison with the oracle's own estimate (its sketch, its Householder QR, its
final pass) runs at the dense workload size (the oracle finishes it in seconds), on the whole
CSR 8e6 x 1024 workload and on a 4,194,304-row prefix of the CSR 8e7 x 1024 workload (the
oracle takes a few minutes of host time for each: about 1e9 FP64 Gaussian draws for G).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import estimator as E, rng as orng

from ._gpu import lev_module, max_rel, to_dev, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    return lev_module()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle(0)


def _sketch_entries(col_of, n, s, m, seed, js, cs):
    """A~[j, c] for j in js, c in cs from the oracle streams; col_of(c) -> dense column c of A (FP64)."""
    b, sign = orng.bucket_and_sign(n, s, seed)
    out = np.zeros((len(js), len(cs)))
    Grows = np.stack([orng.gaussian_sketch_block(m, s, seed, 0, s)[j] for j in js]) if m * s <= 2 ** 26 else None
    for ci, c in enumerate(cs):
        Bc = np.zeros(s)
        np.add.at(Bc, b, sign * col_of(c))
        for ji, j in enumerate(js):
            if Grows is not None:
                g = Grows[ji]
            else:
                idx = np.uint64(j) * np.uint64(s) + np.arange(s, dtype=np.uint64)
                g = orng.sketch_gaussian(seed, idx, m)
            out[ji, ci] = g @ Bc
    return out


def _abs_entries(col_of, n, s, m, seed, js, cs):
    b, _ = orng.bucket_and_sign(n, s, seed)
    out = np.zeros((len(js), len(cs)))
    for ci, c in enumerate(cs):
        Bc = np.zeros(s)
        np.add.at(Bc, b, np.abs(col_of(c)))
        for ji, j in enumerate(js):
            idx = np.uint64(j) * np.uint64(s) + np.arange(s, dtype=np.uint64)
            out[ji, ci] = np.abs(orng.sketch_gaussian(seed, idx, m)) @ Bc
    return out


def _check_qr(At, perm, R, r, rs):
    d = perm.size
    assert sorted(perm.tolist()) == list(range(d))
    Rk = R[:r, :r]
    assert np.all(np.diag(Rk) > 0)
    assert np.all(np.tril(Rk, -1) == 0)
    # (A~ P)^T (A~ P) = R^T R on sampled entries of the leading block
    AP = At.astype(np.float64)[:, perm[:r]]
    for _ in range(40):
        a, c = rs.integers(0, r, 2)
        lhs = AP[:, a] @ AP[:, c]
        rhs = R[:, a] @ R[:, c]
        scale = np.linalg.norm(AP[:, a]) * np.linalg.norm(AP[:, c])
        assert abs(lhs - rhs) <= 1e-5 * scale


def _rows_theta(C, rows, Mf):
    """theta~ of the given CSR rows from Mfull, FP64, straight from the CSR arrays."""
    M64 = Mf.astype(np.float64)
    out = np.empty(len(rows))
    for t, i in enumerate(rows):
        a, b = C.row_ptr[i], C.row_ptr[i + 1]
        y = C.val[a:b].astype(np.float64) @ M64[C.col[a:b]]
        out[t] = y @ y
    return out


def _run_stages(L, h, p, sketch, final, d, m, k):
    import torch
    At = torch.empty((m, d), dtype=torch.float32, device="cuda")
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    R = torch.empty((d, d), dtype=torch.float64, device="cuda")
    Mf = torch.empty((d, k), dtype=torch.float32, device="cuda")
    sketch(At)
    r = L.lev_rrqr(h, At, p.tau, perm, R)
    d_rank = torch.tensor([r], dtype=torch.int64, device="cuda")
    L.lev_omega_factor(h, R, perm, d_rank, d, k, p.seed, L.LEV_OMEGA_REDUCED, Mf)
    theta = final(Mf)
    torch.cuda.synchronize()
    return to_np(At), to_np(perm), to_np(R), r, to_np(Mf), theta


def test_dense_1e6x256_end_to_end(L, h):
    """Dense 1e6 x 256 of rank 200 in the bench configuration: rank, pivots and every theta~
    against the oracle's own FP64 estimate (split-BF16 sketch and final pass: 1e-4)."""
    cfg = W.CONFIGS["dense_1e6x256_rank200"]
    A = W.dense_lowrank_skewed(cfg["n"], cfg["d"], cfg["rank"], seed=cfg["data_seed"])
    theta, r, perm = L.estimate(to_dev(A), s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"],
                                sketch_prec="bf16x3", final_prec="bf16x3", handle=h)
    e = E.estimate(A.astype(np.float64), cfg["s"], cfg["m"], cfg["k"], cfg["tau"], cfg["seed"])
    assert r == e.rank == 200
    assert np.array_equal(to_np(perm)[:r], e.perm[:r])
    assert max_rel(to_np(theta), e.theta) <= 1e-4


def test_csr_8e6x1024(L, h):
    """CSR 8e6 x 1024 (8 nnz/row, 1% rows with 256), s = 262144, m = 4096, k = 256, full rank."""
    import torch
    cfg = W.CONFIGS["csr_8e6x1024"]
    n, d, s, m, k = cfg["n"], cfg["d"], cfg["s"], cfg["m"], cfg["k"]
    C = W.csr_uniform(n, d, seed=cfg["data_seed"])
    rp, cl, vl = to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val)
    p = L.make_params(s=s, m=m, k=k, tau=cfg["tau"], seed=cfg["seed"], sketch_prec="bf16x3")
    theta_t = torch.empty(n, device="cuda")
    At, perm, R, r, Mf, _ = _run_stages(
        L, h, p, lambda out: L.lev_sketch_csr(h, rp, cl, vl, n, d, p, out),
        lambda Mf_: (L.lev_final_csr(h, rp, cl, vl, n, d, Mf_, "fp32", theta_t), to_np(theta_t))[1], d, m, k)
    theta = to_np(theta_t)
    rs = np.random.default_rng(0)
    Asp = sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=(n, d)).tocsc()
    col_of = lambda c: Asp[:, c].toarray().ravel()
    js, cs = rs.integers(0, m, 3), rs.integers(0, d, 3)
    want = _sketch_entries(col_of, n, s, m, cfg["seed"], js, cs)
    scale = _abs_entries(col_of, n, s, m, cfg["seed"], js, cs)
    assert np.all(np.abs(At[np.ix_(js, cs)] - want) <= 1e-4 * scale)
    assert r == d
    _check_qr(At, perm, R, r, rs)
    rows = rs.integers(0, n, 2000)
    assert max_rel(theta[rows], _rows_theta(C, rows, Mf)) <= 1e-5


_GRAM_CACHE = {}


def _host_gram(C, n, d):
    """A^T A of a CSR matrix in FP64 on the host: rows with more than 32 entries densified through
    a BLAS product, the others as a scipy sparse product (kept for the module: two tests use the
    CSR 8e6 x 1024 matrix)."""
    key = (n, d, C.nnz, float(C.val[:64].astype(np.float64).sum()))
    A = sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=(n, d))
    if key not in _GRAM_CACHE:
        heavy = np.diff(C.row_ptr) > 32
        Ah = A[np.flatnonzero(heavy)].toarray()
        Al = A[np.flatnonzero(~heavy)]
        _GRAM_CACHE.clear()
        _GRAM_CACHE[key] = Ah.T @ Ah + (Al.T @ Al).toarray()
    return A, _GRAM_CACHE[key]


def test_csr_8e6x1024_srht(L, h):
    """The CSR 8e6 x 1024 workload with the SRHT after the CountSketch (t = 36,864 rows, the
    size of the quoted SRHT theorem at d = 1024, s = 262,144): full rank, sampled theta~ from the
    GPU's Mfull, sum theta~ = ||A Mfull||_F^2 = tr(Mfull^T (A^T A) Mfull) exactly (host FP64 Gram),
    and, loosely, against the Gaussian-Wishart expectation r m / (m - r - 1) (exact only when F S
    is an isometry on range(A); the composed sketch distorts it by a few percent)."""
    import torch
    cfg = W.CONFIGS["csr_8e6x1024"]
    n, d, s, m, k = cfg["n"], cfg["d"], cfg["s"], cfg["m"], cfg["k"]
    C = W.csr_uniform(n, d, seed=cfg["data_seed"])
    rp, cl, vl = to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val)
    p = L.make_params(s=s, m=m, k=k, tau=cfg["tau"], seed=cfg["seed"], sketch_prec="bf16x3", srht_t=36864)
    theta_t = torch.empty(n, device="cuda")
    At, perm, R, r, Mf, _ = _run_stages(
        L, h, p, lambda out: L.lev_sketch_csr(h, rp, cl, vl, n, d, p, out),
        lambda Mf_: (L.lev_final_csr(h, rp, cl, vl, n, d, Mf_, "fp32", theta_t), to_np(theta_t))[1], d, m, k)
    theta = to_np(theta_t)
    assert r == d
    rs = np.random.default_rng(2)
    _check_qr(At, perm, R, r, rs)
    rows = rs.integers(0, n, 2000)
    assert max_rel(theta[rows], _rows_theta(C, rows, Mf)) <= 1e-5
    got = float(theta.astype(np.float64).sum())
    _, B = _host_gram(C, n, d)
    Mf64 = Mf.astype(np.float64)
    assert abs(got / float(np.sum(Mf64 * (B @ Mf64))) - 1) < 1e-5
    want_sum = r * m / (m - r - 1)
    assert abs(got / want_sum - 1) < 0.1


def test_csr_8e6x1024_exact(L, h):
    """Alg. 7 on the CSR 8e6 x 1024 workload (lev_exact_csr): full rank, the scores sum to the
    rank (trace of the hat matrix), 0 <= theta <= 1, and 2,000 sampled rows against
    a_K B^{-1} a_K^T with B = A^T A formed on the host in FP64 (rows with more than 32 entries
    densified through a BLAS product, the others as a scipy sparse product)."""
    import scipy.linalg as sla
    import torch
    cfg = W.CONFIGS["csr_8e6x1024"]
    n, d, s, m, k = cfg["n"], cfg["d"], cfg["s"], cfg["m"], cfg["k"]
    C = W.csr_uniform(n, d, seed=cfg["data_seed"])
    p = L.make_params(s=s, m=m, k=k, tau=cfg["tau"], seed=cfg["seed"], sketch_prec="bf16x3")
    theta_t = torch.empty(n, device="cuda")
    perm_t = torch.empty(d, dtype=torch.int32, device="cuda")
    r = L.lev_exact_csr(h, to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val), n, d, p, theta_t, perm_t)
    theta = to_np(theta_t).astype(np.float64)
    assert r == d
    assert abs(theta.sum() - d) < 1e-4 * d
    assert theta.min() >= 0 and theta.max() <= 1 + 1e-5
    A, B = _host_gram(C, n, d)
    cf = sla.cho_factor(B)
    rows = np.random.default_rng(4).integers(0, n, 2000)
    Ar = A[rows].toarray()
    want = np.einsum("ij,ij->i", Ar, sla.cho_solve(cf, Ar.T).T)
    assert max_rel(theta[rows], want) <= 1e-5
    assert L.lev_device_status(h) == 0


def test_csr_8e7x1024_rank1014(L, h):
    """CSR 8e7 x 1024, ~12 nnz/row (~1e9 nnz), column j + 512 = 2 x column j for j < 10:
    rank exactly 1014, no dependent pair both selected, sampled sketch entries and theta~."""
    import torch
    cfg = W.CONFIGS["csr_8e7x1024_rank1014"]
    n, d, s, m, k = cfg["n"], cfg["d"], cfg["s"], cfg["m"], cfg["k"]
    C = W.csr_dup_columns(n, d, seed=cfg["data_seed"])
    rp, cl, vl = to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val)
    p = L.make_params(s=s, m=m, k=k, tau=cfg["tau"], seed=cfg["seed"], sketch_prec="bf16x3")
    theta_t = torch.empty(n, device="cuda")
    At, perm, R, r, Mf, _ = _run_stages(
        L, h, p, lambda out: L.lev_sketch_csr(h, rp, cl, vl, n, d, p, out),
        lambda Mf_: (L.lev_final_csr(h, rp, cl, vl, n, d, Mf_, "fp32", theta_t), to_np(theta_t))[1], d, m, k)
    theta = to_np(theta_t)
    assert r == 1014
    sel = set(perm[:r].tolist())
    for j in range(10):
        assert not ({j, j + 512} <= sel)
    # dependent columns of the sketch stay exactly dependent (sums in a fixed order)
    for j in range(10):
        assert np.array_equal(At[:, j + 512], 2.0 * At[:, j])
    rs = np.random.default_rng(1)
    _check_qr(At, perm, R, r, rs)
    rows = rs.integers(0, n, 2000)
    assert max_rel(theta[rows], _rows_theta(C, rows, Mf)) <= 1e-5
    # sum_i theta~_i = ||A_K R_11^{-1} Omega||_F^2; with an m-row Gaussian stage its expectation is
    # r m / (m - r - 1) (mean of the inverse Wishart), about 1348 here
    got = float(theta.astype(np.float64).sum())
    _, B = _host_gram(C, n, d)
    Mf64 = Mf.astype(np.float64)
    assert abs(got / float(np.sum(Mf64 * (B @ Mf64))) - 1) < 1e-5
    want_sum = r * m / (m - r - 1)
    assert abs(got / want_sum - 1) < 0.1


def _first_pivot_difference(gp, e, r):
    """First step t at which the GPU's pivot differs from the oracle's, with the relative gap of the
    two columns' squared trailing norms at that step (from the oracle's R, pivot order)."""
    diff = np.flatnonzero(gp[:r] != e.perm[:r])
    if diff.size == 0:
        return None
    t = int(diff[0])
    pos = {int(c): q for q, c in enumerate(e.perm)}
    R = e.R

    def trailing(c):
        q = pos[int(c)]
        return float(np.sum(R[t:q + 1, q] ** 2)) if q < R.shape[0] else float(np.sum(R[t:, q] ** 2))

    a, b = trailing(e.perm[t]), trailing(gp[t])
    return t, int(e.perm[t]), int(gp[t]), abs(a - b) / a


# Relative gap of two squared trailing norms below which the pivot choice between the two columns is
# a tie at the precision of the split-BF16 sketch (each product carried to about 2^-16 of itself): the
# GPU's sketch and the oracle's FP64 sketch may order such a pair differently, and either order is a
# correct greedy pivot.
PIVOT_TIE = 1e-5


def _csr_end_to_end(L, h, C, cfg):
    """The GPU estimate of CSR C (split-BF16 sketch, FP32 CSR final pass) against the oracle's FP64
    estimate on the same matrix: rank; pivots equal on the first r positions up to the first step
    where the two candidates' squared trailing norms tie to within PIVOT_TIE (from there the greedy
    paths may part, both correct); theta~ on every row against the oracle run at the GPU's pivots."""
    import torch
    n, d = C.shape
    s, m, k, tau, seed = cfg["s"], cfg["m"], cfg["k"], cfg["tau"], cfg["seed"]
    p = L.make_params(s=s, m=m, k=k, tau=tau, seed=seed, sketch_prec="bf16x3")
    theta_t = torch.empty(n, device="cuda")
    perm_t = torch.empty(d, dtype=torch.int32, device="cuda")
    r = L.lev_estimate_csr(h, to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val), n, d, p, theta_t, perm_t)
    theta, gp = to_np(theta_t).astype(np.float64), to_np(perm_t)
    A = sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=(n, d))
    e = E.estimate(A, s, m, k, tau, seed)
    assert r == e.rank
    d0 = _first_pivot_difference(gp, e, r)
    if d0 is not None:
        e = E.estimate(A, s, m, k, tau, seed, forced_perm=gp, forced_rank=r, Atilde=e.Atilde)
    assert max_rel(theta, e.theta) <= 1e-4
    assert d0 is None or d0[3] <= PIVOT_TIE, \
        "first pivot difference at step %d: oracle column %d, GPU column %d, gap %.2e" % d0
    return r


def test_csr_8e6x1024_end_to_end_against_oracle(L, h):
    """The CSR 8e6 x 1024 workload end to end against the oracle's own FP64 estimate (its sketch,
    its Householder QR, its final pass): rank, the 1,024 pivots in order up to the first tie at the
    sketch's precision (one measured run: equal through step 696, then two columns whose squared
    trailing norms differ by 3.4e-9 relative), theta~ on all 8e6 rows within the 1e-4 bar of the
    split-BF16 sketch with the FP32 CSR final pass."""
    cfg = W.CONFIGS["csr_8e6x1024"]
    C = W.csr_uniform(cfg["n"], cfg["d"], seed=cfg["data_seed"])
    assert _csr_end_to_end(L, h, C, cfg) == cfg["d"]


def test_csr_8e7x1024_prefix_end_to_end_against_oracle(L, h):
    """The first 4,194,304 rows of the CSR 8e7 x 1024 workload (the generator draws in blocks of 2^20
    rows, so these are exactly the matrix's first rows), with its s, m, k: rank 1,014 from the ten
    doubled column pairs, the pivots in order and theta~ on every row against the oracle's FP64
    estimate; d = 1,024 takes the same pivoted-Cholesky route as the whole matrix."""
    cfg = W.CONFIGS["csr_8e7x1024_rank1014"]
    C = W.csr_dup_columns(4 << 20, cfg["d"], seed=cfg["data_seed"])
    assert _csr_end_to_end(L, h, C, cfg) == 1014
