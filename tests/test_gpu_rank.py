"""GPU parity of the rank decisions beyond the diagonal test (lev_rrqr_select; LEV_RANK_SVD,
LEV_SRRQR) against the FP64 oracle (oracle/rank.py).

* Singular values: the one-sided Jacobi SVD of R against LAPACK's singular values of the same FP32
  sketch (read exactly into FP64): |sigma_gpu - sigma| <= 1e-9 sigma_1 (FP64 Householder QR and a
  Jacobi tolerance of 1e-12 on the cosines, far inside that).
* SVD rank: equal to the oracle's count on matrices with a clear gap at tau; the paper's
  fixed_svd_1e7 case (gap of 10 at the cutoff 10^-6.5) end to end with the FP32 sketch.
* Strong RRQR: the GPU's final columns satisfy max rho <= phi (rho from the oracle's QR of the
  same sketch, 1e-6 relative slack for the Gram route's rounding); the swap sequence from the same
  start equals the oracle's; theta~ at the GPU's columns within 1e-4 of the oracle.
"""
import numpy as np
import pytest

import workloads as W
from oracle import estimator as E, rank as K
from oracle.linalg import pivoted_qr

from ._gpu import lev_module, max_rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    return lev_module()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle(0)


def _select(L, h, At, **kw):
    import torch
    m, d = At.shape
    p = L.make_params(s=64, m=m, k=8, **kw)
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    R = torch.empty((d, d), dtype=torch.float64, device="cuda")
    sig = torch.empty(d, dtype=torch.float64, device="cuda") if kw.get("rank_svd") else None
    r, swaps = L.lev_rrqr_select(h, to_dev(At), p, perm, R, sigma=sig)
    torch.cuda.synchronize()
    return r, swaps, to_np(perm), to_np(R), (to_np(sig) if sig is not None else None)


@pytest.mark.parametrize("m,d", [(120, 60), (1024, 256), (2000, 1000), (301, 77)])
def test_singular_values_and_rank(L, h, m, d):
    rs = np.random.default_rng(d)
    k = d // 2
    sig = np.concatenate([np.logspace(0, -3, k), np.logspace(-6, -8, d - k)])
    At = W.fixed_svd(m, d, sig, seed=d).astype(np.float32)
    r, swaps, perm, R, s_gpu = _select(L, h, At, tau=1e-4, rank_svd=True)
    s_ref = K.singular_values(At.astype(np.float64))
    assert np.all(np.abs(s_gpu - s_ref) <= 1e-9 * s_ref[0])
    assert r == K.rank_svd(s_ref, 1e-4) == k
    ref = pivoted_qr(At.astype(np.float64), 0.0)
    assert np.array_equal(perm[:r], ref.perm[:r])
    assert swaps == 0


def test_svd_rank_finds_fixed_svd_1e7(L, h):
    """Sec. 7.2's matrix: singular values 1 (15), 1e-6 (15), 1e-7 (30), cutoff 10^-6.5: rank 30 from
    the singular values of the sketch (FP32 sketch arithmetic). kappa(R11) is about 1e6 at the
    selected columns, so theta~ moves by O(u_32 kappa) with the FP32 rounding of the sketch and
    of the final pass; it is checked against the oracle's steps 4-7 on the GPU's own sketch, within
    10 u_32 kappa(R11)."""
    import torch
    sig = np.concatenate([np.ones(15), np.full(15, 1e-6), np.full(30, 1e-7)])
    A = W.fixed_svd(50000, 60, sig, seed=7).astype(np.float32)
    cfg = dict(s=5 * (60 * 60 + 60), m=120, k=64, tau=10 ** -6.5, seed=3)
    p = L.make_params(sketch_prec="fp32", final_prec="fp32", rank_svd=True, **cfg)
    dA = to_dev(A)
    theta = torch.empty(A.shape[0], device="cuda")
    perm = torch.empty(60, dtype=torch.int32, device="cuda")
    r = L.lev_estimate_dense(h, dA, p, theta, perm)
    assert r == 30
    At = torch.empty((120, 60), device="cuda")
    L.lev_sketch_dense(h, dA, p, At)
    e = E.estimate(A.astype(np.float64), cfg["s"], cfg["m"], cfg["k"], cfg["tau"], cfg["seed"],
                   Atilde=to_np(At).astype(np.float64), forced_perm=to_np(perm), forced_rank=30)
    kappa = np.linalg.cond(e.R[:, :30])
    assert kappa > 1e5
    assert max_rel(to_np(theta), e.theta) <= 10 * 2.0 ** -24 * kappa


@pytest.mark.parametrize("m,d,k_true,phi", [(200, 48, 24, 1.01), (1024, 256, 200, 1.05), (600, 150, 149, 1.001)])
def test_srrqr_swaps_match_oracle(L, h, m, d, k_true, phi):
    rs = np.random.default_rng(m)
    sig = np.concatenate([np.logspace(0, -3, k_true), np.logspace(-7, -9, d - k_true)])
    At = (W.fixed_svd(m, d, sig, seed=m + 1) @ np.diag(np.exp(rs.standard_normal(d)))).astype(np.float32)
    A64 = At.astype(np.float64)
    r, swaps, perm, R, _ = _select(L, h, At, tau=1e-5, srrqr_phi=phi)
    assert r == k_true
    rho = K.srrqr_measures(K.r_factor(A64, perm), r)[0]
    assert rho.max() <= phi * (1 + 1e-6)
    start = pivoted_qr(A64, 1e-5)
    assert start.rank == r
    operm, rhos, _ = K.srrqr(A64, r, phi, start.perm)
    assert swaps == len(rhos)
    # the selected columns in order; the others in any order (the forced factor lists them its way)
    assert np.array_equal(perm[:r], operm[:r]) and set(perm[r:].tolist()) == set(operm[r:].tolist())
    # R rows < r are the QR factor of A~ at the final columns
    Rref = K.r_factor(A64, perm)[:r]
    assert np.abs(R[:r] - Rref).max() <= 1e-8 * np.abs(Rref).max()


def test_estimate_with_srrqr_matches_oracle(L, h):
    import torch
    A = W.dense_lowrank_skewed(40000, 64, 40, seed=11)
    cfg = dict(s=8192, m=256, k=64, tau=1e-5, seed=4)
    p = L.make_params(sketch_prec="bf16x3", final_prec="fp32", rank_svd=True, srrqr_phi=1.2, **cfg)
    theta = torch.empty(A.shape[0], device="cuda")
    perm = torch.empty(64, dtype=torch.int32, device="cuda")
    r = L.lev_estimate_dense(h, to_dev(A), p, theta, perm)
    assert r == 40
    e = E.estimate(A.astype(np.float64), cfg["s"], cfg["m"], cfg["k"], cfg["tau"], cfg["seed"],
                   forced_perm=to_np(perm), forced_rank=r)
    assert max_rel(to_np(theta), e.theta) <= 1e-4
    assert L.lev_device_status(h) == 0


def test_rank_rules_reject_bad_arguments(L, h):
    import torch
    At = to_dev(W.dense_gaussian(64, 16, 0).astype(np.float32))
    perm = torch.empty(16, dtype=torch.int32, device="cuda")
    R = torch.empty((16, 16), dtype=torch.float64, device="cuda")
    sig = torch.empty(16, dtype=torch.float64, device="cuda")
    for kw, s_ in [(dict(srrqr_phi=0.5), None), (dict(), sig)]:
        with pytest.raises(L.LevError) as e:
            L.lev_rrqr_select(h, At, L.make_params(s=64, m=64, k=8, **kw), perm, R, sigma=s_)
        assert e.value.code == L.LEV_EINVAL
    Z = torch.zeros((64, 16), device="cuda")
    r, _ = L.lev_rrqr_select(h, Z, L.make_params(s=64, m=64, k=8, rank_svd=True), perm, R, sigma=sig)
    assert r == 0
    r, sw = L.lev_rrqr_select(h, At, L.make_params(s=64, m=64, k=8, rank_svd=True, srrqr_phi=2.0), perm, R)
    assert r == 16 and sw == 0                           # full rank: nothing to swap
