"""GPU parity: every stage of the CUDA path against the FP64 oracle (through the C ABI).

Tolerances (FP32 path):
* sketch entries: |A~_gpu - A~_oracle| <= 2e-5 * (|G| |S| |A|) entrywise -- FP32
  sums of at most a few thousand terms per split, fixed order;
* pivots bit-exact on the first r positions, rank bit-exact;
* R: relative 1e-10 (FP64 on both sides, different summation order);
* Mfull: relative 1e-6 to the FP64 solve rounded once to FP32 (the GPU solve runs in double-float
  arithmetic, about 48 bits, for d <= 1024);
* final pass with identical inputs: relative 1e-5 per row (FP32 products);
* end to end theta~: max relative error 1e-4 against the oracle's FP64 theta~.
"""
import numpy as np
import pytest

import workloads as W
from oracle import estimator as E, exact as X, linalg as OL

from ._gpu import lev_module, max_rel, sketch_abs_scale, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    return lev_module()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle(0)


# ---------------------------------------------------------------- sketch

@pytest.mark.parametrize("n,d,s,m", [(5000, 24, 1024, 96), (3001, 37, 700, 150), (20000, 256, 2048, 1024),
                                     (777, 130, 5000, 300), (1, 4, 3, 8)])
def test_sketch_dense_parity(L, h, n, d, s, m):
    import torch
    A = W.dense_gaussian(n, d, seed=n + d).astype(np.float32)
    p = L.make_params(s=s, m=m, seed=5)
    At = torch.empty((m, d), dtype=torch.float32, device="cuda")
    L.lev_sketch_dense(h, to_dev(A), p, At)
    torch.cuda.synchronize()
    A64 = A.astype(np.float64)
    want = E.sketch(A64, s, m, 5)
    scale = sketch_abs_scale(A64, s, m, 5)
    err = np.abs(to_np(At) - want)
    assert np.all(err <= 2e-5 * scale + 1e-30), float(np.max(err / (scale + 1e-30)))


# Relative error of one entry of G as each form's Gaussian stage applies it: the FP32 draw is a few
# FP32 ulp of the FP64 one; the operand then carries it to 2^-16 (BF16 hi + lo), 2^-11 (TF32) or
# 2^-8 (BF16) of itself.
G_ENTRY_TOL = {"fp32": 1e-6, "bf16x3": 2e-5, "tf32": 1e-3, "bf16": 4e-3}


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "tf32", "bf16"])
def test_gaussian_entries_match_oracle_draws(L, h, prec):
    """The entries of G entry by entry: with A = I (n = d) column i of S A is sigma_i e_{h(i)}, so
    column i of A~ = G S A is sigma_i G[:, h(i)], one column of G read back through the sketch.
    Against the oracle's FP64 Box-Muller draws (stream 2) divided by sqrt(m): every entry within
    the form's relative bound, including draws near 0 (u1 near 1, or cos near its zero)."""
    import torch
    from oracle import rng as orng
    d, s, m, seed = 512, 65536, 256, 7
    A = np.eye(d, dtype=np.float32)
    p = L.make_params(s=s, m=m, seed=seed, sketch_prec=prec)
    At = torch.empty((m, d), dtype=torch.float32, device="cuda")
    L.lev_sketch_dense(h, to_dev(A), p, At)
    b, sign = orng.bucket_and_sign(d, s, seed)
    idx = np.arange(m, dtype=np.uint64)[:, None] * np.uint64(s) + b.astype(np.uint64)[None, :]
    want = orng.sketch_gaussian(seed, idx, m) * sign[None, :]
    got = to_np(At).astype(np.float64)
    rel = np.abs(got - want) / np.abs(want)
    assert np.all(rel <= G_ENTRY_TOL[prec]), (prec, float(rel.max()))
    assert np.median(rel) < G_ENTRY_TOL[prec] / 2


SKETCH_TC_TOL = {"bf16x3": 1e-4, "tf32": 2e-3, "bf16": 1.6e-2}


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "bf16"])
@pytest.mark.parametrize("n,d,s,m", [(5000, 24, 1024, 96), (3001, 36, 700, 150), (20000, 256, 2048, 1024),
                                     (777, 300, 5000, 300), (1, 4, 3, 8)])
def test_sketch_dense_tensor_core_parity(L, h, prec, n, d, s, m):
    """tcgen05 Gaussian stage: |A~_gpu - A~_oracle| <= tol (|G| |S| |A|) entrywise, tol from the
    operand rounding of the form (2^-16 split BF16, 2^-11 TF32, 2^-8 BF16) and FP32 accumulation."""
    import torch
    A = W.dense_gaussian(n, d, seed=n + d + 1).astype(np.float32)
    p = L.make_params(s=s, m=m, seed=7, sketch_prec=prec)
    At = torch.full((m, d), float("nan"), dtype=torch.float32, device="cuda")
    L.lev_sketch_dense(h, to_dev(A), p, At)
    torch.cuda.synchronize()
    A64 = A.astype(np.float64)
    want = E.sketch(A64, s, m, 7)
    scale = sketch_abs_scale(A64, s, m, 7)
    err = np.abs(to_np(At) - want)
    assert np.all(err <= SKETCH_TC_TOL[prec] * scale + 1e-30), float(np.max(err / (scale + 1e-30)))
    assert L.lev_device_status(h) == 0


def test_estimate_tensor_core_sketch_and_final(L, h):
    """Split-BF16 Gaussian stage and split-BF16 final pass: rank exact, theta~ within 1e-4."""
    A = W.dense_lowrank_skewed(60000, 64, 40, seed=21)
    cfg = dict(s=8192, m=256, k=128, tau=1e-4, seed=3)
    theta, r, perm = L.estimate(to_dev(A), handle=h, sketch_prec="bf16x3", final_prec="bf16x3", **cfg)
    e = _oracle_estimate(A, cfg)
    assert r == e.rank == 40
    assert np.array_equal(to_np(perm)[:r], e.perm[:r])
    assert max_rel(to_np(theta), e.theta) <= 1e-4


def test_sketch_dense_strided_and_repeatable(L, h):
    import torch
    A = W.dense_gaussian(4099, 64, seed=3).astype(np.float32)
    big = torch.zeros((4099, 80), dtype=torch.float32, device="cuda")
    big[:, :64] = to_dev(A)
    view = big[:, :64]
    p = L.make_params(s=512, m=128, seed=9)
    out1 = torch.empty((128, 64), device="cuda")
    out2 = torch.empty((128, 64), device="cuda")
    L.lev_sketch_dense(h, view, p, out1)
    L.lev_sketch_dense(h, to_dev(A), p, out2)
    torch.cuda.synchronize()
    assert torch.equal(out1, out2)             # fixed summation order: bit-identical
    want = E.sketch(A.astype(np.float64), 512, 128, 9)
    assert np.max(np.abs(to_np(out1) - want)) <= 2e-5 * np.max(sketch_abs_scale(A.astype(np.float64), 512, 128, 9))


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("n,d,s,m", [(20000, 256, 2048, 1024), (777, 300, 5000, 300), (3000, 1000, 3000, 256),
                                     (5000, 24, 1024, 96), (1, 4, 3, 8)])
def test_sketch_operand_written_by_countsketch_is_the_transposed_one(L, h, prec, n, d, s, m):
    """BF16 forms: the CountSketch writes the Gaussian stage's operand itself (blocked by 64
    buckets) when A allows 16-byte loads; a view of A 4 bytes off that alignment takes the other
    route (FP32 B, then the transpose kernel). Both round the same sums the same way, so A~ is
    bit-identical."""
    import torch
    A = W.dense_gaussian(n, d, seed=n + d).astype(np.float32)
    p = L.make_params(s=s, m=m, seed=5, sketch_prec=prec)
    flat = torch.zeros(n * d + 1, dtype=torch.float32, device="cuda")
    flat[1:] = to_dev(A).reshape(-1)
    off_view = flat[1:].view(n, d)                       # data pointer 4 bytes past a 16-byte boundary
    assert off_view.data_ptr() % 16 != 0
    out_fused = torch.full((m, d), float("nan"), device="cuda")
    out_plain = torch.full((m, d), float("nan"), device="cuda")
    L.lev_sketch_dense(h, to_dev(A), p, out_fused)
    L.lev_sketch_dense(h, off_view, p, out_plain)
    torch.cuda.synchronize()
    assert torch.equal(out_fused, out_plain)
    assert L.lev_device_status(h) == 0


def test_sketch_csr_parity(L, h):
    import torch
    C = W.csr_uniform(6000, 200, nnz_per_row=5, heavy_frac=0.02, heavy_nnz=60, seed=4)
    p = L.make_params(s=1500, m=400, seed=2)
    At = torch.empty((400, 200), device="cuda")
    L.lev_sketch_csr(h, to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val), 6000, 200, p, At)
    torch.cuda.synchronize()
    dense = C.to_dense()
    want = E.sketch(dense, 1500, 400, 2)
    scale = sketch_abs_scale(dense, 1500, 400, 2)
    assert np.all(np.abs(to_np(At) - want) <= 2e-5 * scale + 1e-30)


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("n,d,s,m,heavy", [(6000, 200, 1500, 400, 60), (3000, 1024, 2000, 256, 300),
                                           (50, 8, 3, 8, 8)])
def test_sketch_csr_operand_matches_dense_of_the_same_matrix(L, h, prec, n, d, s, m, heavy):
    """BF16 forms: the dense CountSketch writes the Gaussian stage's operand itself, the CSR one
    writes FP32 B for the transpose kernel. A bucket's sum runs over the same rows in the same order
    on both paths, and each entry adds sign x value once (the dense kernel's zeros leave its sums
    unchanged), and both round B to the operand the same way, so the CSR sketch equals the dense
    sketch of the densified matrix bit for bit; and both are within the form's bound of the
    oracle."""
    import torch
    C = W.csr_uniform(n, d, nnz_per_row=5, heavy_frac=0.02, heavy_nnz=heavy, seed=n + d)
    p = L.make_params(s=s, m=m, seed=6, sketch_prec=prec)
    dense = C.to_dense()
    out_csr = torch.full((m, d), float("nan"), device="cuda")
    out_dense = torch.full((m, d), float("nan"), device="cuda")
    L.lev_sketch_csr(h, to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val), n, d, p, out_csr)
    L.lev_sketch_dense(h, to_dev(dense.astype(np.float32)), p, out_dense)
    torch.cuda.synchronize()
    assert torch.equal(out_csr, out_dense)
    want = E.sketch(dense, s, m, 6)
    scale = sketch_abs_scale(dense, s, m, 6)
    assert np.all(np.abs(to_np(out_csr) - want) <= SKETCH_TC_TOL[prec] * scale + 1e-30)
    assert L.lev_device_status(h) == 0


# ---------------------------------------------------------------- rrqr + omega

def _rank_deficient_sketch(m, d, r, seed):
    rs = np.random.default_rng(seed)
    X_ = rs.standard_normal((m, r)) @ rs.standard_normal((r, d))
    X_ *= np.exp(rs.standard_normal(d))[None, :]
    return X_.astype(np.float32)


@pytest.mark.parametrize("m,d,r,tau", [(96, 24, 24, 1e-5), (300, 64, 40, 1e-5), (1024, 256, 200, 1e-4),
                                       (50, 70, 50, 1e-5), (8, 1, 1, 1e-5), (700, 513, 300, 1e-5),
                                       (96, 24, 24, 1e-9), (300, 64, 64, 1e-9), (1024, 512, 400, 1e-5),
                                       (2048, 1024, 900, 1e-5), (60, 20, 20, 1e-5), (1024, 256, 256, 1e-5)])
def test_rrqr_parity(L, h, m, d, r, tau):
    """Pivots and rank bit-exact, R close to the oracle's Householder R.

    d <= 1024 with tau >= 1e-6 runs the Gram route (pivoted Cholesky of A~^T A~ on one
    cooperative grid, FP64), whose R differs from Householder's by O(u kappa(R_11)^2); the other
    cases run the Householder kernel (O(u kappa))."""
    import torch
    At = _rank_deficient_sketch(m, d, r, seed=m + d)
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    R = torch.empty((d, d), dtype=torch.float64, device="cuda")
    rank = L.lev_rrqr(h, to_dev(At), tau, perm, R)
    q = OL.pivoted_qr(At.astype(np.float64), tau)
    assert rank == q.rank == min(r, m, d)
    gp = to_np(perm)
    assert np.array_equal(gp[:rank], q.perm[:rank])
    assert sorted(gp.tolist()) == list(range(d))
    assert np.all(np.diff(gp[rank:]) > 0)               # the rest in increasing order
    gR = to_np(R)
    Rg = gR[:rank]
    Rw = np.zeros_like(Rg)                               # oracle R, columns moved to the GPU order
    colpos = {c: t for t, c in enumerate(gp)}
    for t, c in enumerate(q.perm):
        Rw[:, colpos[c]] = q.R[:, t]
    assert np.all(np.diag(Rg[:, :rank]) > 0)
    kappa = np.linalg.cond(Rw[:, :rank])
    tol = max(1e-10, 50 * 2.0 ** -53 * kappa ** 2)
    assert np.max(np.abs(Rg - Rw)) <= tol * np.max(np.abs(Rw)), (kappa, np.max(np.abs(Rg - Rw)) / np.max(np.abs(Rw)))
    assert np.all(gR[rank:] == 0)


def test_rrqr_rank_zero(L, h):
    import torch
    perm = torch.empty(5, dtype=torch.int32, device="cuda")
    R = torch.empty((5, 5), dtype=torch.float64, device="cuda")
    assert L.lev_rrqr(h, torch.zeros((12, 5), device="cuda"), 1e-5, perm, R) == 0
    assert to_np(perm).tolist() == list(range(5))
    assert np.all(to_np(R) == 0)


@pytest.mark.parametrize("k,identity", [(64, False), (100, False), (0, True)])
def test_omega_factor_parity(L, h, k, identity):
    import torch
    m, d, r = 300, 64, 40
    At = _rank_deficient_sketch(m, d, r, seed=7)
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    R = torch.empty((d, d), dtype=torch.float64, device="cuda")
    rank = L.lev_rrqr(h, to_dev(At), 1e-5, perm, R)
    kk = d if identity else k
    Mf = torch.empty((d, kk), dtype=torch.float32, device="cuda")
    d_rank = torch.tensor([rank], dtype=torch.int64, device="cuda")
    L.lev_omega_factor(h, R, perm, d_rank, d, kk, 13, L.LEV_OMEGA_IDENTITY if identity else 0, Mf)
    torch.cuda.synchronize()
    R64, gp = to_np(R), to_np(perm)
    M = E.omega_factor(R64[:rank, :rank], kk, 13, omega_identity=identity)
    if identity:
        M = np.hstack([M, np.zeros((rank, kk - rank))])
    want = E.m_full(M, gp, d)
    got = to_np(Mf).astype(np.float64)
    assert np.max(np.abs(got - want)) <= 1e-6 * np.max(np.abs(want))
    assert np.all(got[gp[rank:]] == 0)


@pytest.mark.parametrize("d,r,k", [(1024, 1000, 24), (1100, 1050, 8)])
def test_omega_factor_wide(L, h, d, r, k):
    """d = 1024 (the double-float solve with 32 rows a lane, its largest form) and d > 1024 (the
    FP64 kernel that draws Omega itself): a synthetic upper-triangular R with a dominant diagonal,
    a random pivot order."""
    import torch
    rs = np.random.default_rng(d)
    R = np.triu(rs.standard_normal((d, d)) * 0.05) + np.diag(1.0 + rs.random(d))
    gp = rs.permutation(d).astype(np.int32)
    Mf = torch.empty((d, k), dtype=torch.float32, device="cuda")
    d_rank = torch.tensor([r], dtype=torch.int64, device="cuda")
    L.lev_omega_factor(h, to_dev(R), to_dev(gp), d_rank, d, k, 21, 0, Mf)
    torch.cuda.synchronize()
    want = E.m_full(E.omega_factor(R[:r, :r], k, 21), gp, d)
    got = to_np(Mf).astype(np.float64)
    assert np.max(np.abs(got - want)) <= 1e-6 * np.max(np.abs(want))
    assert np.all(got[gp[r:]] == 0)


def test_omega_cache_follows_seed_and_shape(L, h):
    """The handle's Omega cache is keyed by (seed, d, k): alternating seeds and k give the oracle's
    M every time."""
    import torch
    rs = np.random.default_rng(3)
    d, r = 48, 40
    R = np.triu(rs.standard_normal((d, d)) * 0.1) + np.diag(1.0 + rs.random(d))
    gp = np.arange(d, dtype=np.int32)
    d_rank = torch.tensor([r], dtype=torch.int64, device="cuda")
    for seed, k in [(13, 16), (14, 16), (13, 16), (13, 24)]:
        Mf = torch.empty((d, k), dtype=torch.float32, device="cuda")
        L.lev_omega_factor(h, to_dev(R), to_dev(gp), d_rank, d, k, seed, 0, Mf)
        torch.cuda.synchronize()
        want = E.m_full(E.omega_factor(R[:r, :r], k, seed), gp, d)
        got = to_np(Mf).astype(np.float64)
        assert np.max(np.abs(got - want)) <= 1e-6 * np.max(np.abs(want))


@pytest.mark.parametrize("d,r,k", [(256, 200, 256), (64, 20, 64), (300, 50, 100), (1024, 500, 600),
                                   (40, 39, 40), (256, 256, 256), (256, 200, 128)])
def test_omega_factor_reduced(L, h, d, r, k):
    """LEV_OMEGA_REDUCED: for r < k, row perm[p] of Mfull holds row p of W = R_11^{-1} L_r in the
    first r columns and zeros after, with L_r the Cholesky factor (lower, positive diagonal) of
    Omega_r Omega_r^T for the oracle's first r rows of Omega; for r >= k it is M = R_11^{-1} Omega_r.
    Either way Mfull Mfull^T is the oracle's M M^T, the only product theta~ depends on."""
    import torch
    from scipy.linalg import solve_triangular
    rs = np.random.default_rng(d + r + k)
    R = np.triu(rs.standard_normal((d, d)) * 0.05) + np.diag(1.0 + rs.random(d))
    gp = rs.permutation(d).astype(np.int32)
    Mf = torch.empty((d, k), dtype=torch.float32, device="cuda")
    d_rank = torch.tensor([r], dtype=torch.int64, device="cuda")
    L.lev_omega_factor(h, to_dev(R), to_dev(gp), d_rank, d, k, 31, L.LEV_OMEGA_REDUCED, Mf)
    torch.cuda.synchronize()
    got = to_np(Mf).astype(np.float64)
    M = E.m_full(E.omega_factor(R[:r, :r], k, 31), gp, d)
    if r < k:
        Om = E.omega_factor(np.eye(r), k, 31)                 # Omega_r
        W = solve_triangular(R[:r, :r], np.linalg.cholesky(Om @ Om.T), lower=False)
        want = np.zeros((d, k))
        want[gp[:r], :r] = W
    else:
        want = M
    assert np.max(np.abs(got - want)) <= 1e-6 * np.max(np.abs(want))
    assert np.all(got[gp[r:]] == 0)
    P, Pw = got @ got.T, M @ M.T
    assert np.max(np.abs(P - Pw)) <= 2e-6 * np.max(np.abs(Pw))


# ---------------------------------------------------------------- final pass

@pytest.mark.parametrize("n,d,k,lda", [(10007, 256, 256, 256), (999, 37, 100, 37), (5000, 64, 512, 80),
                                       (64, 16, 8, 16), (1, 4, 4, 4)])
def test_final_dense_parity(L, h, n, d, k, lda):
    import torch
    rs = np.random.default_rng(n)
    A = rs.standard_normal((n, lda)).astype(np.float32)
    Mf = (rs.standard_normal((d, k)) / np.sqrt(d)).astype(np.float32)
    Mf[rs.random(d) < 0.2] = 0.0
    Ad = to_dev(A)[:, :d]
    theta = torch.empty(n, device="cuda")
    L.lev_final_dense(h, Ad, to_dev(Mf), "fp32", theta)
    torch.cuda.synchronize()
    want = np.sum((A[:, :d].astype(np.float64) @ Mf.astype(np.float64)) ** 2, axis=1)
    assert max_rel(to_np(theta), want) <= 1e-5


TC_TOL = {"bf16": 1e-2, "tf32": 2e-3, "bf16x3": 5e-5}


@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3"])
@pytest.mark.parametrize("n,d,k,lda", [(10007, 256, 256, 256), (999, 36, 100, 36), (5000, 64, 200, 80),
                                       (1, 4, 4, 4), (300, 256, 17, 256), (129, 128, 256, 132),
                                       (777, 37, 64, 40), (999, 37, 100, 37), (500, 250, 33, 251)])
def test_final_dense_tensor_core_parity(L, h, prec, n, d, k, lda):
    """tcgen05 forms of the final pass against the FP64 product of the same FP32 inputs; d need not
    be a multiple of 4, and a row stride that TMA cannot take (lda % 4 != 0) goes through a padded copy."""
    import torch
    rs = np.random.default_rng(n + d + k)
    A = rs.standard_normal((n, lda)).astype(np.float32)
    Mf = (rs.standard_normal((d, k)) / np.sqrt(d)).astype(np.float32)
    Mf[rs.random(d) < 0.2] = 0.0
    theta = torch.full((n,), float("nan"), device="cuda")
    L.lev_final_dense(h, to_dev(A)[:, :d], to_dev(Mf), prec, theta)
    torch.cuda.synchronize()
    want = np.sum((A[:, :d].astype(np.float64) @ Mf.astype(np.float64)) ** 2, axis=1)
    assert max_rel(to_np(theta), want) <= TC_TOL[prec]
    assert L.lev_device_status(h) == 0


def test_final_dense_tensor_core_rejects_unsupported(L, h):
    import torch
    A = torch.zeros((10, 300), device="cuda")
    with pytest.raises(L.LevError) as e:
        L.lev_final_dense(h, A, torch.zeros((300, 8), device="cuda"), "bf16", torch.empty(10, device="cuda"))
    assert e.value.code == L.LEV_EINVAL


def test_final_csr_parity(L, h):
    import torch
    C = W.csr_uniform(5003, 300, nnz_per_row=6, heavy_frac=0.01, heavy_nnz=200, seed=8)
    rs = np.random.default_rng(1)
    Mf = (rs.standard_normal((300, 256)) / 17).astype(np.float32)
    theta = torch.empty(5003, device="cuda")
    L.lev_final_csr(h, to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val), 5003, 300, to_dev(Mf), "fp32", theta)
    torch.cuda.synchronize()
    want = np.sum((C.to_dense() @ Mf.astype(np.float64)) ** 2, axis=1)
    assert max_rel(to_np(theta), want) <= 1e-5


@pytest.mark.parametrize("k", [256, 64])
def test_final_csr_both_forms_of_lemma1(L, h, k):
    """Rows of 0..40 entries straddle the switch between the second form of Lemma 1 (a P a^T for
    rows of <= 32 entries) and the first (||a Mfull||^2); columns unsorted, repeated (they add up)
    and, on some rows, outside [0, d) (they count as zero)."""
    import torch
    rs = np.random.default_rng(k)
    n, d = 6001, 120
    lens = rs.integers(0, 41, size=n)
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = rs.integers(0, d, size=row_ptr[-1]).astype(np.int32)
    col[rs.random(col.size) < 0.01] = d + 5                      # out of range
    val = rs.standard_normal(row_ptr[-1]).astype(np.float32)
    Mf = (rs.standard_normal((d, k)) / np.sqrt(k)).astype(np.float32)
    theta = torch.full((n,), float("nan"), device="cuda")
    L.lev_final_csr(h, to_dev(row_ptr), to_dev(col), to_dev(val), n, d, to_dev(Mf), "fp32", theta)
    torch.cuda.synchronize()
    ok = col < d
    rows = np.repeat(np.arange(n), lens)
    Adense = np.zeros((n, d))
    np.add.at(Adense, (rows[ok], col[ok]), val[ok].astype(np.float64))
    want = np.sum((Adense @ Mf.astype(np.float64)) ** 2, axis=1)
    got = to_np(theta).astype(np.float64)
    assert np.all(got[lens == 0] == 0)
    assert max_rel(got, want) <= 1e-5


# ---------------------------------------------------------------- end to end

def _oracle_estimate(A32, cfg):
    return E.estimate(A32.astype(np.float64), cfg["s"], cfg["m"], cfg["k"], cfg["tau"], cfg["seed"])


def test_estimate_small_dense_workload(L, h):
    cfg = W.CONFIGS["dense_2000x20_f64"]
    A = W.dense_gaussian(cfg["n"], cfg["d"], cfg["data_seed"]).astype(np.float32)
    theta, r, perm = L.estimate(to_dev(A), s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"],
                                handle=h)
    e = _oracle_estimate(A, cfg)
    assert r == e.rank == 20
    assert np.array_equal(to_np(perm)[:r], e.perm[:r])
    assert max_rel(to_np(theta), e.theta) <= 1e-4


def test_estimate_lowrank_skewed(L, h):
    A = W.dense_lowrank_skewed(60000, 64, 40, seed=21)
    cfg = dict(s=8192, m=256, k=128, tau=1e-4, seed=3)
    theta, r, perm = L.estimate(to_dev(A), handle=h, **cfg)
    e = _oracle_estimate(A, cfg)
    assert r == e.rank == 40
    assert np.array_equal(to_np(perm)[:r], e.perm[:r])
    assert max_rel(to_np(theta), e.theta) <= 1e-4


# Unit roundoff of the operand rounding of each form (A and Mfull are rounded once each).
FORM_U = {"bf16": 2.0 ** -9, "tf32": 2.0 ** -11, "bf16x3": 2.0 ** -17}


def _final_pass_condition(A64, perm, r, M):
    """c_i = sum_q |y_iq| (|A_iK| |M|)_q / sum_q y_iq^2: the rounding amplification of row i."""
    AK = A64[:, perm[:r]]
    Y = AK @ M
    Yabs = np.abs(AK) @ np.abs(M)
    return np.sum(np.abs(Y) * Yabs, axis=1) / np.sum(Y * Y, axis=1)


@pytest.mark.parametrize("prec,tol", [("bf16", None), ("tf32", 5e-3), ("bf16x3", 1e-4)])
def test_estimate_lowrank_skewed_tensor_core(L, h, prec, tol):
    """End to end with a tensor-core final pass. TF32 must meet the mixed-precision bar
    (5e-3) and BF16X3 the split bar (1e-4); plain BF16 must stay within its rounding
    bound 4 u c_i per row (u = 2^-9, c_i the row's amplification) plus the FP32 sketch error."""
    A = W.dense_lowrank_skewed(60000, 64, 40, seed=21)
    cfg = dict(s=8192, m=256, k=128, tau=1e-4, seed=3)
    theta, r, perm = L.estimate(to_dev(A), handle=h, final_prec=prec, **cfg)
    e = _oracle_estimate(A, cfg)
    assert r == e.rank == 40
    got = to_np(theta).astype(np.float64)
    rel = np.abs(got - e.theta) / e.theta
    c = _final_pass_condition(A.astype(np.float64), e.perm, r, e.M)
    assert np.all(rel <= 4 * FORM_U[prec] * c + 1e-4)
    if tol is not None:
        assert rel.max() <= tol


def test_estimate_csr(L, h):
    import torch
    C = W.csr_uniform(40000, 128, nnz_per_row=8, heavy_frac=0.01, heavy_nnz=64, seed=6)
    cfg = dict(s=8192, m=512, k=64, tau=1e-5, seed=4)
    p = L.make_params(**cfg)
    theta = torch.empty(40000, device="cuda")
    perm = torch.empty(128, dtype=torch.int32, device="cuda")
    r = L.lev_estimate_csr(h, to_dev(C.row_ptr), to_dev(C.col), to_dev(C.val), 40000, 128, p, theta, perm)
    import scipy.sparse as sp
    Asp = sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=C.shape)
    e = E.estimate(Asp, **cfg)
    assert r == e.rank == 128
    assert np.array_equal(to_np(perm)[:r], e.perm[:r])
    assert max_rel(to_np(theta), e.theta) <= 1e-4


def test_identity_modes_give_exact_leverage(L, h):
    A = W.dense_gaussian(3000, 12, seed=5).astype(np.float32)
    theta, r, _ = L.estimate(to_dev(A), tau=1e-6, sketch_identity=True, omega_identity=True, handle=h)
    th, rx = X.exact_leverage_qr(A.astype(np.float64), 1e-6)
    assert r == rx == 12
    assert max_rel(to_np(theta), th) <= 1e-4
    assert abs(float(to_np(theta).sum()) - 12) < 1e-3


def test_forced_pivots_match_oracle(L, h):
    import torch
    A = W.dense_gaussian(5000, 16, seed=8).astype(np.float32)
    forced = np.random.default_rng(0).permutation(16).astype(np.int32)
    p = L.make_params(s=2048, m=64, k=32, seed=1, perm_in=to_dev(forced), rank_in=10)
    theta = torch.empty(5000, device="cuda")
    perm = torch.empty(16, dtype=torch.int32, device="cuda")
    r = L.lev_estimate_dense(h, to_dev(A), p, theta, perm)
    e = E.estimate(A.astype(np.float64), 2048, 64, 32, 1e-5, 1, forced_perm=forced, forced_rank=10)
    assert r == 10
    assert np.array_equal(to_np(perm)[:10], forced[:10])
    assert max_rel(to_np(theta), e.theta) <= 1e-4


def test_scale_invariance_bit_exact(L, h):
    A = W.dense_gaussian(7000, 32, seed=9).astype(np.float32)
    t1, r1, p1 = L.estimate(to_dev(A), s=1024, m=128, k=64, seed=2, handle=h)
    t2, r2, p2 = L.estimate(to_dev(2.0 * A), s=1024, m=128, k=64, seed=2, handle=h)
    assert r1 == r2 and np.array_equal(to_np(p1), to_np(p2))
    assert np.array_equal(to_np(t1), to_np(t2))


def test_zero_rows_and_rank_zero(L, h):
    A = W.dense_gaussian(3000, 8, seed=10).astype(np.float32)
    A[[0, 17, 2999]] = 0
    theta, r, _ = L.estimate(to_dev(A), s=512, m=32, k=16, seed=3, handle=h)
    assert r == 8 and np.all(to_np(theta)[[0, 17, 2999]] == 0)
    theta0, r0, _ = L.estimate(to_dev(np.zeros((100, 6), np.float32)), s=64, m=24, k=8, handle=h)
    assert r0 == 0 and np.all(to_np(theta0) == 0)


def test_host_buffers_match_device_path(L, h):
    import torch
    A = W.dense_gaussian(9000, 48, seed=11).astype(np.float32)
    p = L.make_params(s=2048, m=192, k=64, seed=6)
    th_dev = torch.empty(9000, device="cuda")
    r1 = L.lev_estimate_dense(h, to_dev(A), p, th_dev)
    A_host = torch.from_numpy(A).pin_memory()
    th_host = torch.empty(9000, dtype=torch.float32).pin_memory()
    r2 = L.lev_estimate_dense(h, A_host, p, th_host)
    A_page = torch.from_numpy(A.copy())
    th_page = torch.empty(9000, dtype=torch.float32)
    r3 = L.lev_estimate_dense(h, A_page, p, th_page)
    assert r1 == r2 == r3 == 48
    assert torch.equal(th_dev.cpu(), th_host) and torch.equal(th_host, th_page)


def test_host_async_pipelined_calls(L, h):
    """LEV_HOST_ASYNC: three enqueued calls on different host inputs (the stage buffers alternate,
    so the third copy must wait for the first call's kernels), then one synchronisation; each
    theta equals the device path's bit for bit, and so does a synchronous call afterwards. The
    host inputs are overwritten only after the synchronisation."""
    import torch
    As = [W.dense_gaussian(12000, 40, seed=20 + i).astype(np.float32) for i in range(3)]
    As[1] *= np.exp(np.random.default_rng(5).standard_normal(40)).astype(np.float32)[None, :]
    p_sync = L.make_params(s=4096, m=160, k=64, seed=9, sketch_prec="bf16x3", final_prec="bf16x3")
    p_async = L.make_params(s=4096, m=160, k=64, seed=9, sketch_prec="bf16x3", final_prec="bf16x3",
                            host_async=True)
    want = []
    for A in As:
        t = torch.empty(12000, device="cuda")
        assert L.lev_estimate_dense(h, to_dev(A), p_sync, t) == 40
        want.append(t.cpu())
    hosts = [torch.from_numpy(A).pin_memory() for A in As]
    outs = [torch.full((12000,), float("nan")).pin_memory() for _ in As]
    for Ah, th in zip(hosts, outs):
        L.lev_estimate_dense(h, Ah, p_async, th, want_rank=False)
    torch.cuda.synchronize()
    assert L.lev_device_status(h) == 0
    for th, w in zip(outs, want):
        assert torch.equal(th, w)
    for Ah in hosts:
        Ah.zero_()
    th = torch.empty(12000).pin_memory()
    assert L.lev_estimate_dense(h, torch.from_numpy(As[2]).pin_memory(), p_sync, th) == 40
    assert torch.equal(th, want[2])


def test_rrqr_timing_diagnostics(L, h):
    """lev_set_timing / lev_rrqr_timing: positive durations for both kernels of the Gram route,
    gram 0-width on the Householder route, EINVAL when timing is off."""
    import torch
    At = to_dev(_rank_deficient_sketch(300, 64, 40, seed=1))
    perm = torch.empty(64, dtype=torch.int32, device="cuda")
    R = torch.empty((64, 64), dtype=torch.float64, device="cuda")
    L.lev_set_timing(h, True)
    try:
        with pytest.raises(L.LevError):
            L.lev_rrqr_timing(h)                          # no QR since timing was enabled
        assert L.lev_rrqr(h, At, 1e-5, perm, R) == 40
        g_ms, f_ms = L.lev_rrqr_timing(h)
        assert g_ms > 0 and f_ms > 0
        assert L.lev_rrqr(h, At, 1e-9, perm, R) >= 40     # tau < 1e-6: Householder route (FP32 noise ranks)
        g_ms, f_ms = L.lev_rrqr_timing(h)
        assert g_ms >= 0 and f_ms > 0
    finally:
        L.lev_set_timing(h, False)
    with pytest.raises(L.LevError) as e:
        L.lev_rrqr_timing(h)
    assert e.value.code == L.LEV_EINVAL


def test_fresh_handle_first_call(L):
    """First call on a new handle: every scratch buffer is freshly allocated."""
    A = W.dense_gaussian(2000, 20, seed=0).astype(np.float32)
    for _ in range(2):
        h2 = L.Handle(0)
        theta, r, perm = L.estimate(to_dev(A), s=1600, m=80, k=64, tau=1e-10, seed=0, handle=h2)
        h2.close()
        assert r == 20
        e = E.estimate(A.astype(np.float64), 1600, 80, 64, 1e-10, 0)
        assert max_rel(to_np(theta), e.theta) <= 1e-4


def test_invalid_arguments(L, h):
    import torch
    A = torch.zeros((10, 4), device="cuda")
    theta = torch.empty(10, device="cuda")
    with pytest.raises(L.LevError) as e:
        L.lev_estimate_dense(h, A, L.make_params(s=0, eps=1.5), theta)
    assert e.value.code == L.LEV_EINVAL
    with pytest.raises(L.LevError):
        L.lev_final_dense(h, A, torch.zeros((4, 8), device="cuda"), 9, theta)
    assert L.lev_device_status(h) == 0


def test_prepare_builds_the_caches_and_changes_no_result(L):
    """lev_prepare builds G, the bucket permutation and Omega ahead of the first call: the estimate
    that follows is bit-identical to one on a fresh handle, and the prepared handle already holds
    at least the G pair (two m x s BF16 images)."""
    import torch
    A = to_dev(W.dense_gaussian(6000, 48, 3).astype(np.float32))
    p = L.make_params(s=4096, m=192, k=32, tau=1e-6, seed=8, sketch_prec="bf16x3", final_prec="bf16x3")
    h1, h2 = L.Handle(0), L.Handle(0)
    try:
        L.lev_prepare(h1, 6000, 48, p)
        assert L.lev_workspace_bytes(h1) >= 64 + 2 * 192 * 4096 * 2
        t1 = torch.empty(6000, device="cuda")
        t2 = torch.empty(6000, device="cuda")
        r1 = L.lev_estimate_dense(h1, A, p, t1)
        r2 = L.lev_estimate_dense(h2, A, p, t2)
        assert r1 == r2 == 48
        assert torch.equal(t1, t2)
        with pytest.raises(L.LevError) as e:
            L.lev_prepare(h1, 6000, 48, L.make_params(s=0, eps=2.0))
        assert e.value.code == L.LEV_EINVAL
    finally:
        h1.close()
        h2.close()


def test_workspace_bytes_counts_scratch_and_caches(L):
    """lev_workspace_bytes: the status word on a fresh handle; after an estimate at least the cached
    G (the BF16 hi + lo pair, two m x s images); unchanged by a second call of the same shapes
    (buffers only grow)."""
    import torch
    h = L.Handle(0)
    try:
        assert L.lev_workspace_bytes(h) == 64
        A = to_dev(W.dense_gaussian(4096, 32, 1).astype(np.float32))
        p = L.make_params(s=2048, m=128, k=16, tau=1e-8, seed=2, sketch_prec="bf16x3", final_prec="bf16x3")
        theta = torch.empty(4096, device="cuda")
        assert L.lev_estimate_dense(h, A, p, theta) == 32
        b1 = L.lev_workspace_bytes(h)
        assert b1 >= 64 + 2 * 128 * 2048 * 2
        L.lev_estimate_dense(h, A, p, theta)
        assert L.lev_workspace_bytes(h) == b1
    finally:
        h.close()
