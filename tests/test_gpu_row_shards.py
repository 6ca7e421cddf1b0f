"""Row shards on the GPU: block sketches (rows hashed by global index) against the oracle, their
sum against the whole matrix's sketch, the sharded estimate against the oracle, and two processes
on one GPU joined by a gloo all-reduce of the sketch.

Tolerances. A block's sketch: within c |G| |S_block| |A_block| entrywise (c as in the sketch
parity tests: 3e-5 FP32, 1e-4 split BF16). The sum of the blocks against the unsharded GPU sketch:
the same bound on the whole |G| |S| |A| (each bucket's FP32 sum is cut into partial sums: a
reassociation). The estimate: rank and pivots exact, theta~ within 1e-4 of the oracle at the
same pivots (the FP32 bar).
"""
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import estimator as E

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


@pytest.mark.parametrize("prec,c", [("fp32", 3e-5), ("bf16x3", 1e-4)])
@pytest.mark.parametrize("srht_t", [0, 1024])
def test_block_sketches_match_oracle_and_sum(L, h, prec, c, srht_t):
    import torch
    n, d, s, m, seed = 300_001, 96, 4096, 384, 13
    A = W.dense_heavy_rows(n, d, seed=8)
    A64 = A.astype(np.float64)
    p = L.make_params(s=s, m=m, k=64, seed=seed, sketch_prec=prec, srht_t=srht_t)
    dA = to_dev(A)
    whole = torch.empty((m, d), device="cuda")
    L.lev_sketch_dense(h, dA, p, whole)
    total = torch.zeros((m, d), device="cuda")
    for rank in range(3):
        row0, rows = L.row_shard(n, 3, rank)
        part = torch.empty((m, d), device="cuda")
        L.sketch_shard(h, dA[row0:row0 + rows], p, row0, n, part)
        if srht_t == 0:
            want = E.sketch(A64[row0:row0 + rows], s, m, seed, row0=row0)
            scale = sketch_abs_scale(A64[row0:row0 + rows], s, m, seed, row0=row0)
            assert np.all(np.abs(to_np(part).astype(np.float64) - want) <= c * scale + 1e-30)
        total += part
    torch.cuda.synchronize()
    if srht_t == 0:
        scale = sketch_abs_scale(A64, s, m, seed)
        assert np.all(np.abs(to_np(total).astype(np.float64) - to_np(whole)) <= 2 * c * scale + 1e-30)
    want = E.sketch(A64, s, m, seed, srht_t=srht_t)
    err = np.abs(to_np(total).astype(np.float64) - want).max() / np.abs(want).max()
    assert err <= 1e-4


def test_sharded_dense_estimate_matches_oracle(L, h):
    import torch
    n, d, rank_A = 200_003, 64, 40
    cfg = dict(s=8192, m=256, k=128, tau=1e-5, seed=21)
    A = W.dense_lowrank_skewed(n, d, rank_A, seed=9)
    p = L.make_params(sketch_prec="bf16x3", final_prec="fp32", **cfg)
    dA = to_dev(A)
    At = torch.zeros((cfg["m"], d), device="cuda")
    blocks = [L.row_shard(n, 4, r) for r in range(4)]
    for row0, rows in blocks:                      # the all-reduce, emulated in a fixed order
        part = torch.empty_like(At)
        L.sketch_shard(h, dA[row0:row0 + rows], p, row0, n, part)
        At += part
    thetas, perms = [], []
    for row0, rows in blocks:
        th, r, perm = L.finish_shard(h, dA[row0:row0 + rows], p, At, cfg["k"])
        assert r == rank_A
        thetas.append(to_np(th))
        perms.append(to_np(perm))
    assert all(np.array_equal(perms[0], q) for q in perms)
    theta = np.concatenate(thetas)
    ref_theta, ref_r, ref_perm = L.estimate(dA, sketch_prec="bf16x3", final_prec="fp32", handle=h, **cfg)
    assert ref_r == rank_A and np.array_equal(to_np(ref_perm)[:rank_A], perms[0][:rank_A])
    e = E.estimate(A.astype(np.float64), cfg["s"], cfg["m"], cfg["k"], cfg["tau"], cfg["seed"],
                   forced_perm=perms[0], forced_rank=rank_A)
    assert max_rel(theta, e.theta) <= 1e-4
    assert max_rel(theta, to_np(ref_theta)) <= 1e-4


def test_sharded_csr_estimate_matches_oracle(L, h):
    import torch
    n, d = 90_001, 128
    C = W.csr_uniform(n, d, nnz_per_row=6, heavy_frac=0.01, heavy_nnz=96, seed=12)
    cfg = dict(s=16384, m=512, k=64, tau=1e-5, seed=4)
    p = L.make_params(sketch_prec="bf16x3", final_prec="fp32", **cfg)
    At = torch.zeros((cfg["m"], d), device="cuda")
    blocks = [L.row_shard(n, 3, r) for r in range(3)]

    def block_csr(row0, rows):
        a, b = C.row_ptr[row0], C.row_ptr[row0 + rows]
        return (to_dev(C.row_ptr[row0:row0 + rows + 1] - a), to_dev(C.col[a:b]), to_dev(C.val[a:b]), rows, d)

    for row0, rows in blocks:
        part = torch.empty_like(At)
        L.sketch_shard(h, None, p, row0, n, part, csr=block_csr(row0, rows))
        At += part
    thetas = []
    for row0, rows in blocks:
        th, r, perm = L.finish_shard(h, None, p, At, cfg["k"], csr=block_csr(row0, rows))
        thetas.append(to_np(th))
    Asp = sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=(n, d))
    e = E.estimate(Asp, cfg["s"], cfg["m"], cfg["k"], cfg["tau"], cfg["seed"], forced_perm=to_np(perm), forced_rank=r)
    assert r == d
    assert max_rel(np.concatenate(thetas), e.theta) <= 1e-4


def test_estimate_sharded_single_process_equals_estimate(L, h):
    """Without a process group the sharded call is the whole path on one block: bit-identical."""
    import torch
    n, d = 50_000, 32
    A = to_dev(W.dense_lowrank_skewed(n, d, 20, seed=2))
    cfg = dict(s=4096, m=128, k=64, tau=1e-5, seed=3)
    p = L.make_params(sketch_prec="bf16x3", final_prec="bf16x3", **cfg)
    th, r, perm = L.estimate_sharded(A, p, 0, n, handle=h)
    th2, r2, perm2 = L.estimate(A, sketch_prec="bf16x3", final_prec="bf16x3", handle=h, **cfg)
    assert r == r2 == 20
    assert torch.equal(perm, perm2) and torch.equal(th, th2)


def test_whole_matrix_entry_points_reject_a_shard(L, h):
    import torch
    n, d = 1000, 8
    A = to_dev(W.dense_gaussian(n, d, 0).astype(np.float32))
    theta = torch.empty(n, device="cuda")
    shard = L.make_params(s=256, m=32, k=8, row0=1000, n_total=2000)
    for call in (lambda: L.lev_estimate_dense(h, A, shard, theta),
                 lambda: L.lev_exact_dense(h, A, shard, theta)):
        with pytest.raises(L.LevError) as e:
            call()
        assert e.value.code == L.LEV_EINVAL
    At = torch.empty((32, d), device="cuda")
    with pytest.raises(L.LevError) as e:
        L.lev_sketch_dense(h, A, L.make_params(s=256, m=32, k=8, row0=1500, n_total=2000), At)
    assert e.value.code == L.LEV_EINVAL
    p = L.make_params(s=256, m=32, k=8)
    _, st = L.forward_state(A, p, handle=h)
    with pytest.raises(L.LevError) as e:
        L.lev_backward_dense(h, A, shard, st["Atilde"], st["perm"], st["d_rank"], st["R"], st["Mfull"],
                             torch.ones(n, device="cuda"), torch.empty_like(A))
    assert e.value.code == L.LEV_EINVAL


def _free_port():
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        return sck.getsockname()[1]


_TWO_PROC = dict(n=120_001, d=48, rank=30, s=8192, m=192, k=64, tau=1e-5, seed=17)


def _two_process_rank(rank, world, port, out_dir):
    """One of two processes on cuda:0; they meet only in the host-side gloo all-reduce, never in
    a kernel, so neither waits on the other's launches."""
    import torch
    import torch.distributed as dist
    import paper_2105_11004_gb300 as L
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        c = _TWO_PROC
        A = W.dense_lowrank_skewed(c["n"], c["d"], c["rank"], seed=5)
        row0, rows = L.row_shard(c["n"], world, rank)
        p = L.make_params(s=c["s"], m=c["m"], k=c["k"], tau=c["tau"], seed=c["seed"],
                          sketch_prec="bf16x3", final_prec="fp32")
        h = L.Handle(0)
        th, r, perm = L.estimate_sharded(to_dev(A[row0:row0 + rows]), p, row0, c["n"], handle=h)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), theta=to_np(th), rank=r, perm=to_np(perm), row0=row0)
        h.close()
    finally:
        dist.destroy_process_group()


def test_two_processes_gloo_allreduce(L, tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_two_process_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    c = _TWO_PROC
    res = sorted((np.load(os.path.join(tmp_path, f"rank{r}.npz")) for r in range(2)), key=lambda z: int(z["row0"]))
    assert int(res[0]["rank"]) == int(res[1]["rank"]) == c["rank"]
    assert np.array_equal(res[0]["perm"], res[1]["perm"])
    A = W.dense_lowrank_skewed(c["n"], c["d"], c["rank"], seed=5).astype(np.float64)
    e = E.estimate(A, c["s"], c["m"], c["k"], c["tau"], c["seed"], forced_perm=res[0]["perm"], forced_rank=c["rank"])
    assert max_rel(np.concatenate([z["theta"] for z in res]), e.theta) <= 1e-4
