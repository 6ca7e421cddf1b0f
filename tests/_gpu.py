"""Helpers for the GPU parity tests: the library, device copies, oracle bounds."""
import numpy as np

from oracle import rng as orng


def lev_module():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2105_11004_gb300 as L
    return L


def to_dev(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def to_np(t):
    return t.detach().cpu().numpy()


def sketch_abs_scale(A64, s, m, seed, row0=0):
    """|G| (|S| |A|): the scale that bounds the rounding error of each entry of G S A (A the
    block of rows from global row row0)."""
    n, d = A64.shape
    b, _ = orng.bucket_and_sign(n, s, seed, start=row0)
    Babs = np.zeros((s, d))
    np.add.at(Babs, b, np.abs(A64))
    out = np.zeros((m, d))
    blk = 1 << 14
    for c0 in range(0, s, blk):
        c1 = min(s, c0 + blk)
        out += np.abs(orng.gaussian_sketch_block(m, s, seed, c0, c1)) @ Babs[c0:c1]
    return out


def max_rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nz = b != 0
    assert np.all(a[~nz] == 0), "nonzero where the reference is exactly zero"
    return float(np.max(np.abs(a[nz] - b[nz]) / np.abs(b[nz]))) if nz.any() else 0.0
