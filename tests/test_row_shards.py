"""Row shards on CPU: the oracle's block sketches, the host logic of the sharded path, and its one
collective over world-size-2 gloo.

The CountSketch S is one fixed s x n matrix (Sec. 3.4.3), so for a partition of the rows into
blocks P_p, S A = sum_p S_{:,P_p} A_{P_p,:} (block matrix product), and G (and the SRHT F) act
linearly on S A. The pins: each block's sketch against an explicit S built row by row from the
hash, the sum of the blocks against the whole matrix's sketch, and the sharded estimate (sum of
the block sketches, then Alg. 10's QR and final pass per block) against the unsharded one.
"""
import ctypes
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import estimator as E, rng as orng


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2105_11004_gb300 as L
    return L


def _explicit_S(n, s, seed):
    """S (s x n) entry by entry: column i holds sign_i in row h(i) (the CountSketch definition)."""
    S = np.zeros((s, n))
    for i in range(n):
        b, sg = orng.bucket_and_sign(1, s, seed, start=i)
        S[b[0], i] = sg[0]
    return S


def test_oracle_block_sketch_equals_explicit_columns_of_S():
    n, d, s, seed = 301, 5, 64, 3
    A = W.dense_gaussian(n, d, seed=1)
    S = _explicit_S(n, s, seed)
    for row0, rows in [(0, 100), (100, 150), (250, 51)]:
        got = E.count_sketch(A[row0:row0 + rows], s, seed, row0=row0)
        np.testing.assert_allclose(got, S[:, row0:row0 + rows] @ A[row0:row0 + rows], rtol=0, atol=1e-13)
    # hashing by the local index instead would give another matrix
    assert not np.allclose(E.count_sketch(A[100:250], s, seed), S[:, 100:250] @ A[100:250])


@pytest.mark.parametrize("srht_t", [0, 48])
def test_oracle_block_sketches_sum_to_whole(srht_t):
    n, d, s, m, seed = 2003, 12, 128, 40, 7
    A = W.dense_heavy_rows(n, d, seed=2).astype(np.float64)
    whole = E.sketch(A, s, m, seed, srht_t=srht_t)
    cuts = [0, 700, 701, 1500, n]
    parts = sum(E.sketch(A[a:b], s, m, seed, srht_t=srht_t, row0=a) for a, b in zip(cuts[:-1], cuts[1:]))
    np.testing.assert_allclose(parts, whole, rtol=0, atol=1e-12 * np.abs(whole).max())


def test_oracle_sharded_estimate_equals_unsharded_csr():
    n, d, s, m, k, tau, seed = 6000, 40, 2048, 160, 32, 1e-6, 9
    C = W.csr_uniform(n, d, nnz_per_row=5, heavy_frac=0.02, heavy_nnz=30, seed=3)
    A = sp.csr_matrix((C.val.astype(np.float64), C.col, C.row_ptr), shape=(n, d))
    whole = E.estimate(A, s, m, k, tau, seed)
    cuts = [0, 1999, 4000, n]
    At = sum(E.sketch(A[a:b], s, m, seed, row0=a) for a, b in zip(cuts[:-1], cuts[1:]))
    thetas = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        e = E.estimate(A[a:b], s, m, k, tau, seed, Atilde=At)
        assert e.rank == whole.rank and np.array_equal(e.perm, whole.perm)
        thetas.append(e.theta)
    np.testing.assert_allclose(np.concatenate(thetas), whole.theta, rtol=1e-10, atol=0)


def test_row_shard_covers_rows_once(L):
    for n, w in [(10, 3), (7, 7), (1_000_003, 8), (5, 1)]:
        blocks = [L.row_shard(n, w, r) for r in range(w)]
        assert blocks[0][0] == 0
        assert all(a + c == b for (a, c), (b, _) in zip(blocks[:-1], blocks[1:]))
        assert blocks[-1][0] + blocks[-1][1] == n
        assert max(c for _, c in blocks) - min(c for _, c in blocks) <= 1
    for bad in [(3, 4, 0), (10, 2, 2), (10, 0, 0)]:
        with pytest.raises(ValueError):
            L.row_shard(*bad)


def test_resolve_sizes_of_a_shard(L):
    """lev_resolve_sizes runs on the host: k follows n_total; bad shards are EINVAL."""
    p = L.make_params(s=4096, m=64, k=0, eps=0.5)
    _, _, k_whole = L.lev_resolve_sizes(p, 8_000_000, 32)
    _, _, k_block = L.lev_resolve_sizes(L.make_params(s=4096, m=64, k=0, eps=0.5, row0=2_000_000,
                                                      n_total=8_000_000), 1_000_000, 32)
    assert k_block == k_whole
    assert k_whole == int(np.ceil(4 * np.log(8e6) / (0.125 - 0.125 / 3)))
    for kw, n in [(dict(row0=5, n_total=10), 6), (dict(row0=-1), 4), (dict(n_total=-3), 4),
                  (dict(row0=1, n_total=10, sketch_identity=True), 4)]:
        with pytest.raises(L.LevError) as e:
            L.lev_resolve_sizes(L.make_params(s=64, m=8, k=4, **kw), n, 4)
        assert e.value.code == L.LEV_EINVAL
    q = L._shard_params(L.make_params(s=64, m=8, k=4, seed=5, tau=1e-3), 7, 99)
    assert (q.s, q.m, q.k, q.seed, q.tau, q.row0, q.n_total) == (64, 8, 4, 5, 1e-3, 7, 99)
    assert ctypes.sizeof(q) == ctypes.sizeof(L.lev_params)


def _free_port():
    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        return sck.getsockname()[1]


def _gloo_rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    import paper_2105_11004_gb300 as L
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        n, d, s, m, k, tau, seed = 4001, 24, 1024, 96, 32, 1e-6, 11
        A = W.dense_lowrank_skewed(n, d, 18, seed=6).astype(np.float64)
        row0, rows = L.row_shard(n, world, rank)
        part = torch.from_numpy(E.sketch(A[row0:row0 + rows], s, m, seed, row0=row0))
        L.allreduce_sketch(part)                                   # the sharded path's exchange
        everyone = [torch.empty_like(part) for _ in range(world)]
        dist.all_gather(everyone, part)
        assert all(torch.equal(everyone[0], x) for x in everyone)  # one summed sketch everywhere
        e = E.estimate(A[row0:row0 + rows], s, m, k, tau, seed, Atilde=part.numpy())
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), theta=e.theta, perm=e.perm, rank=e.rank,
                 row0=row0, At=part.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.slow
def test_gloo_world2_sharded_estimate(L, tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_gloo_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    n, d, s, m, k, tau, seed = 4001, 24, 1024, 96, 32, 1e-6, 11
    A = W.dense_lowrank_skewed(n, d, 18, seed=6).astype(np.float64)
    whole = E.estimate(A, s, m, k, tau, seed)
    res = [np.load(os.path.join(tmp_path, f"rank{r}.npz")) for r in range(world)]
    np.testing.assert_allclose(res[0]["At"], whole.Atilde, rtol=0, atol=1e-12 * np.abs(whole.Atilde).max())
    for r in res:
        assert int(r["rank"]) == whole.rank == 18
        assert np.array_equal(r["perm"], whole.perm)
    theta = np.concatenate([r["theta"] for r in sorted(res, key=lambda z: int(z["row0"]))])
    np.testing.assert_allclose(theta, whole.theta, rtol=1e-9, atol=0)
