"""Run one stage of the estimator on a synthetic case, a few times, for a profiler.

    python -m paper_2105_11004_gb300.stage_runner final --n 262144 --d 256 --k 256 --prec bf16x3
    python -m paper_2105_11004_gb300.stage_runner rrqr --m 1024 --d 256 --rank 200 --tau 1e-4
    python -m paper_2105_11004_gb300.stage_runner sketch --n 262144 --d 256 --s 65536 --m 1024
    python -m paper_2105_11004_gb300.stage_runner backward --n 200000 --d 64 --k 128
    python -m paper_2105_11004_gb300.stage_runner lsqr --n 262144 --d 256
    python -m paper_2105_11004_gb300.stage_runner svd --m 1024 --d 256 --rank 200
    python -m paper_2105_11004_gb300.stage_runner exact_csr --n 1000000 --d 1024
    python -m paper_2105_11004_gb300.stage_runner estimate_csr --n 8000000 --d 1024

Inputs are seeded and synthetic (the generators of the ``workloads`` module); every stage runs
through the C ABI exactly as ``lev_estimate_dense`` runs it. The script prints the CUDA-event time
of the last repetition; under ncu, select the launch with ``-k`` / ``-s`` / ``-c``.
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("stage", choices=["final", "rrqr", "sketch", "backward", "lsqr", "svd", "exact_csr", "estimate_csr"])
    ap.add_argument("--n", type=int, default=262144)
    ap.add_argument("--d", type=int, default=256)
    ap.add_argument("--k", type=int, default=256)
    ap.add_argument("--m", type=int, default=1024)
    ap.add_argument("--s", type=int, default=65536)
    ap.add_argument("--rank", type=int, default=200)
    ap.add_argument("--tau", type=float, default=1e-4)
    ap.add_argument("--prec", default="bf16x3")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=11)
    a = ap.parse_args(argv)

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np
    import torch
    import workloads as W
    import paper_2105_11004_gb300 as L

    h = L.Handle(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(a.reps - 1):
            fn()
        ev0.record()
        fn()
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1)

    if a.stage in ("final", "sketch", "backward"):
        A = torch.from_numpy(W.dense_lowrank_skewed(a.n, a.d, min(a.rank, a.d), seed=a.seed)).cuda()
    if a.stage == "final":
        rs = np.random.default_rng(a.seed)
        Mf = torch.from_numpy((rs.standard_normal((a.d, a.k)) / np.sqrt(a.d)).astype(np.float32)).cuda()
        theta = torch.empty(a.n, device="cuda")
        ms = timed(lambda: L.lev_final_dense(h, A, Mf, a.prec, theta))
    elif a.stage == "sketch":
        p = L.make_params(s=a.s, m=a.m, k=a.k, seed=a.seed, sketch_prec=a.prec)
        At = torch.empty((a.m, a.d), device="cuda")
        ms = timed(lambda: L.lev_sketch_dense(h, A, p, At))
    elif a.stage == "rrqr":
        rs = np.random.default_rng(a.seed)
        X = rs.standard_normal((a.m, a.rank)) @ rs.standard_normal((a.rank, a.d))
        X *= np.exp(rs.standard_normal(a.d))[None, :]
        At = torch.from_numpy(X.astype(np.float32)).cuda()
        perm = torch.empty(a.d, dtype=torch.int32, device="cuda")
        R = torch.empty((a.d, a.d), dtype=torch.float64, device="cuda")
        ms = timed(lambda: L.lev_rrqr(h, At, a.tau, perm, R))
    elif a.stage == "lsqr":
        # Alg. 11 once, then LSQR on A N (each iteration one fused pass over A)
        b = torch.from_numpy(np.random.default_rng(a.seed).standard_normal(a.n).astype(np.float32)).cuda()
        A = torch.from_numpy(W.dense_lowrank_skewed(a.n, a.d, a.d, seed=a.seed)).cuda()
        p = L.make_params(s=a.s, m=4 * a.d, k=8, tau=1e-10, seed=a.seed, sketch_prec="bf16x3")
        N = torch.empty((a.d, a.d), dtype=torch.float64, device="cuda")
        k = L.lev_precondition_dense(h, A, p, N)
        x = torch.zeros(a.d, dtype=torch.float64, device="cuda")
        ms = timed(lambda: L.lev_lsqr_dense(h, A, N, k, b, x, max_iter=200, atol=1e-6, btol=1e-6))
    elif a.stage == "svd":
        rs = np.random.default_rng(a.seed)
        X = rs.standard_normal((a.m, a.rank)) @ rs.standard_normal((a.rank, a.d))
        At = torch.from_numpy(X.astype(np.float32)).cuda()
        p = L.make_params(s=64, m=a.m, k=8, tau=a.tau, seed=a.seed, rank_svd=True)
        perm = torch.empty(a.d, dtype=torch.int32, device="cuda")
        R = torch.empty((a.d, a.d), dtype=torch.float64, device="cuda")
        ms = timed(lambda: L.lev_rrqr_select(h, At, p, perm, R))
    elif a.stage == "exact_csr":
        C = W.csr_uniform(a.n, a.d, seed=a.seed)
        rp, cl, vl = (torch.from_numpy(v).cuda() for v in (C.row_ptr, C.col, C.val))
        p = L.make_params(s=262144, m=4096, k=256, tau=1e-5, seed=a.seed, sketch_prec="bf16x3")
        theta = torch.empty(a.n, device="cuda")
        ms = timed(lambda: L.lev_exact_csr(h, rp, cl, vl, a.n, a.d, p, theta))
    elif a.stage == "estimate_csr":
        # the whole estimate on the CSR workload of the bench (8 entries a row, 1% rows of 256)
        C = W.csr_uniform(a.n, a.d, seed=2)
        rp, cl, vl = (torch.from_numpy(v).cuda() for v in (C.row_ptr, C.col, C.val))
        p = L.make_params(s=262144, m=4096, k=256, tau=1e-5, seed=12, sketch_prec="bf16x3")
        theta = torch.empty(a.n, device="cuda")
        ms = timed(lambda: L.lev_estimate_csr(h, rp, cl, vl, a.n, a.d, p, theta, want_rank=False))
    else:
        p = L.make_params(s=a.s, m=a.m, k=a.k, tau=a.tau, seed=a.seed, sketch_prec="bf16x3", final_prec="bf16x3")
        w = torch.rand(a.n, device="cuda")
        _, st = L.forward_state(A, p, handle=h)
        gA = torch.empty_like(A)
        ms = timed(lambda: L.lev_backward_dense(h, A, p, st["Atilde"], st["perm"], st["d_rank"], st["R"],
                                                st["Mfull"], w, gA))
    print(f"{a.stage}: {ms:.4f} ms (last of {a.reps})", flush=True)
    h.close()


if __name__ == "__main__":
    main()
