"""GPU parity of the backward pass (gradient of sum_i w_i theta~_i) against the FP64 oracle.

The oracle gradient is itself pinned to central finite differences and to the closed
form 2 (I - H) W (A^+)^T (tests/test_oracle_backward.py). Tolerance: max entrywise
error <= 1e-3 of the largest gradient entry (FP32 passes, FP64 small step).
"""
import numpy as np
import pytest

import workloads as W
from oracle import backward as Bk

from ._gpu import lev_module, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    return lev_module()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle(0)


def _gpu_gradient(L, h, A32, w32, **kw):
    import torch
    p = L.make_params(**kw)
    A = to_dev(A32)
    theta, st = L.forward_state(A, p, handle=h)
    g = torch.full(A.shape, float("nan"), device="cuda")
    L.lev_backward_dense(h, A, p, st["Atilde"], st["perm"], st["d_rank"], st["R"], st["Mfull"], to_dev(w32), g)
    torch.cuda.synchronize()
    return to_np(g).astype(np.float64), to_np(st["perm"]), st["rank"], theta


def _rel(g, ref):
    return float(np.max(np.abs(g - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("sketch_prec", ["fp32", "bf16x3", "tf32"])
def test_backward_small_matches_oracle(L, h, sketch_prec):
    A = W.dense_heavy_rows(500, 8, seed=3)
    w = W.uniform_weights(500, seed=4)
    cfg = dict(s=256, m=32, k=16, tau=1e-10, seed=7)
    g, perm, r, _ = _gpu_gradient(L, h, A, w, sketch_prec=sketch_prec, **cfg)
    assert r == 8
    ref = Bk.gradient(A.astype(np.float64), w.astype(np.float64), perm, r, 256, 32, 16, 7)
    # The GPU gradient is the exact adjoint of the GPU forward; a TF32 sketch perturbs that
    # forward by its operand rounding (2^-11 on G and on B), which moves the gradient by a few
    # units of 2^-11 relative to the oracle's exact-sketch gradient.
    tol = 6 * 2.0 ** -11 if sketch_prec == "tf32" else 1e-4
    assert _rel(g, ref) <= tol


def test_backward_identity_mode_is_exact_gradient(L, h):
    """S = I, G = I, Omega = I: the gradient of sum w_i theta_i is 2 (I - H) W (A^+)^T."""
    A = W.dense_heavy_rows(500, 8, seed=3)
    w = W.uniform_weights(500, seed=4)
    g, perm, r, theta = _gpu_gradient(L, h, A, w, tau=1e-10, sketch_identity=True, omega_identity=True)
    assert r == 8
    ref = Bk.exact_gradient(A.astype(np.float64), w.astype(np.float64))
    assert _rel(g, ref) <= 1e-3


def test_backward_strided_input(L, h):
    """A as a column slice with an odd row stride (lda = d + 3): the scalar-load paths of both
    backward passes and of the padded tensor-core final pass, against the oracle."""
    import torch
    n, d = 3000, 20
    A = W.dense_heavy_rows(n, d, seed=12)
    w = W.uniform_weights(n, seed=13)
    Ab = torch.zeros((n, d + 3), dtype=torch.float32, device="cuda")
    Ab[:, :d] = to_dev(A)
    Av = Ab[:, :d]
    p = L.make_params(s=1024, m=80, k=32, tau=1e-8, seed=5, sketch_prec="bf16x3", final_prec="bf16x3")
    theta, st = L.forward_state(Av, p, handle=h)
    g = torch.full((n, d), float("nan"), device="cuda")
    L.lev_backward_dense(h, Av, p, st["Atilde"], st["perm"], st["d_rank"], st["R"], st["Mfull"], to_dev(w), g)
    torch.cuda.synchronize()
    assert st["rank"] == d
    ref = Bk.gradient(A.astype(np.float64), w.astype(np.float64), to_np(st["perm"]), d, 1024, 80, 32, 5)
    assert _rel(to_np(g).astype(np.float64), ref) <= 1e-4


def test_backward_dropped_columns_are_zero(L, h):
    A = W.dense_heavy_rows(3000, 12, seed=5)
    A[:, 9] = 2.0 * A[:, 4]
    w = W.uniform_weights(3000, seed=6)
    g, perm, r, _ = _gpu_gradient(L, h, A, w, s=1024, m=48, k=32, tau=1e-5, seed=2)
    assert r == 11
    assert np.all(g[:, perm[r:]] == 0)
    ref = Bk.gradient(A.astype(np.float64), w.astype(np.float64), perm, r, 1024, 48, 32, 2)
    assert _rel(g, ref) <= 1e-4


def test_backward_full_size_workload(L, h):
    """The 200,000 x 64 backward workload (5% rows x 100, w ~ U(0,1)), s = 16384, m = 256, k = 128."""
    cfg = W.CONFIGS["dense_2e5x64_backward"]
    A = W.dense_heavy_rows(cfg["n"], cfg["d"], seed=cfg["data_seed"])
    w = W.uniform_weights(cfg["n"], seed=cfg["weight_seed"])
    g, perm, r, _ = _gpu_gradient(L, h, A, w, s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"],
                                  sketch_prec="bf16x3")
    assert r == 64
    ref = Bk.gradient(A.astype(np.float64), w.astype(np.float64), perm, r, cfg["s"], cfg["m"], cfg["k"],
                      cfg["seed"])
    assert _rel(g, ref) <= 1e-3


def test_autograd_function(L, h):
    import torch
    A32 = W.dense_heavy_rows(2000, 16, seed=9)
    w32 = W.uniform_weights(2000, seed=10)
    p = L.make_params(s=512, m=64, k=32, tau=1e-8, seed=4)
    A = to_dev(A32).requires_grad_(True)
    theta = L.LevScore.apply(A, p)
    (theta * to_dev(w32)).sum().backward()
    g_auto = to_np(A.grad).astype(np.float64)
    g_direct, perm, r, _ = _gpu_gradient(L, h, A32, w32, s=512, m=64, k=32, tau=1e-8, seed=4)
    assert np.array_equal(g_auto, g_direct)


@pytest.mark.parametrize("sketch_prec,t", [("fp32", 64), ("bf16x3", 64), ("bf16x3", 256)])
def test_backward_srht_matches_oracle(L, h, sketch_prec, t):
    """The SRHT after the CountSketch (t = 256 = s draws many rows twice): the gradient against the
    oracle's, whose SRHT adjoint D H P^T / sqrt(t) is pinned by <F B, Y> = <B, F^T Y> and finite
    differences."""
    A = W.dense_heavy_rows(500, 8, seed=3)
    w = W.uniform_weights(500, seed=4)
    cfg = dict(s=256, m=32, k=16, tau=1e-10, seed=7)
    g, perm, r, _ = _gpu_gradient(L, h, A, w, sketch_prec=sketch_prec, srht_t=t, **cfg)
    assert r == 8
    ref = Bk.gradient(A.astype(np.float64), w.astype(np.float64), perm, r, 256, 32, 16, 7, srht_t=t)
    assert _rel(g, ref) <= 1e-4


def test_backward_srht_full_size_and_repeatable(L, h):
    """The 200,000 x 64 backward workload with an SRHT to t = 2,048 rows: against the oracle, and two
    runs bit-identical (the scatter of repeated draws adds in draw order)."""
    cfg = W.CONFIGS["dense_2e5x64_backward"]
    A = W.dense_heavy_rows(cfg["n"], cfg["d"], seed=cfg["data_seed"])
    w = W.uniform_weights(cfg["n"], seed=cfg["weight_seed"])
    kw = dict(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"], sketch_prec="bf16x3", srht_t=2048)
    g, perm, r, _ = _gpu_gradient(L, h, A, w, **kw)
    g2, _, _, _ = _gpu_gradient(L, h, A, w, **kw)
    assert np.array_equal(g, g2)
    assert r == 64
    ref = Bk.gradient(A.astype(np.float64), w.astype(np.float64), perm, r, cfg["s"], cfg["m"], cfg["k"],
                      cfg["seed"], srht_t=2048)
    assert _rel(g, ref) <= 1e-3

