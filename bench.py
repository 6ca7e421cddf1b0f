"""Benchmark of the rank-revealing leverage-score estimator on one GB300.

One step = one pass of the whole method (Alg. 10) over the dense 1,000,000 x 256
FP32 workload of rank 200 with lognormal(0, 2) row scaling: bucket
permutation, CountSketch, Gaussian stage (s = 65,536, m = 1,024), FP64 pivoted
QR and rank, M = R_11^{-1} Omega (k = 256), fused final pass writing theta~.
The handle caches G (m x s, generated once per seed); every other stage runs
in every step. A (1.02 GB) is larger than L2 (129 MB), so no L2 flush is used.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--sketch-prec fp32|tf32|bf16|bf16x3] [--final-prec ...]
  python bench.py --stage final|rrqr|sketch|backward|lsqr|svd|exact_csr|estimate_csr
                  [--n N --d D --k K --m M --s S --rank R --tau T --prec P --reps K]   (profiling)

Prints one JSON line (rank 0). For N > 1 (torchrun) every rank runs its own
replica on its own GPU (the path is run as replicas; no data is exchanged).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

WORKLOAD = "dense_1e6x256_rank200"
METRIC = "leverage rows/s & HBM GB/s: BF16/TF32-TC vs FP32 path at equal rel err; bwd/fwd"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            pk = json.load(f)
        return pk, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 25 ms in a thread."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "25",
                 "-i", str(device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        sel = [p for (t, p) in self.samples if t0 <= t <= t1]
        if not sel:
            sel = [p for (t, p) in self.samples if t0 - 0.1 <= t <= t1 + 0.1]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[1]) for p in sel if num(p[1]) is not None]
        mx = [num(p[2]) for p in sel if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in sel for i in range(4) if p[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sel),
                "power_w_max": max((num(p[3]) or 0.0) for p in sel)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gpu_numa_placement(device: int):
    """Run this process (and so its pinned host buffers, placed on first touch) on the CPUs local to
    the GPU: the PCI device's NUMA node and CPU list from sysfs. Returns what was found and done."""
    info = {"pci_bus_id": None, "numa_node": None, "cpus": None, "pinned_to_node": False}
    try:
        import torch
        props = torch.cuda.get_device_properties(device)
        bus = getattr(props, "pci_bus_id", None)
        if bus is None:
            uuid = str(getattr(props, "uuid", ""))
            out = subprocess.run(["nvidia-smi", "--query-gpu=uuid,pci.bus_id", "--format=csv,noheader"],
                                 capture_output=True, text=True, timeout=20).stdout
            for line in out.splitlines():
                u, b = [x.strip() for x in line.split(",")]
                if uuid and uuid.replace("GPU-", "") in u:
                    bus = b
        if isinstance(bus, int):
            bus = "%04x:%02x:%02x.0" % (getattr(props, "pci_domain_id", 0), bus, getattr(props, "pci_device_id", 0))
        if bus:
            dom, rest = bus.split(":", 1)
            bus = ("%04x:" % int(dom, 16)) + rest.lower()
            info["pci_bus_id"] = bus
            base = f"/sys/bus/pci/devices/{bus}"
            with open(f"{base}/numa_node") as f:
                node = int(f.read().strip())
            info["numa_node"] = node
            with open(f"{base}/local_cpulist") as f:
                cpus = set()
                for part in f.read().strip().split(","):
                    a, _, b = part.partition("-")
                    cpus.update(range(int(a), int(b or a) + 1))
            allowed = set(os.sched_getaffinity(0))
            use = sorted(cpus & allowed)
            if use and node >= 0:
                os.sched_setaffinity(0, use)
                info["cpus"] = len(use)
                info["pinned_to_node"] = True
    except Exception as e:                       # no sysfs entry (or no permission): leave it as is
        info["error"] = str(e)[:120]
    return info


def host_link(A_host, A_dev, theta_host, theta_dev, reps=3):
    """Pinned host <-> device copy rates on a side stream, CUDA events (best of reps)."""
    import torch
    st = torch.cuda.Stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h2d, d2h = [], []
    for _ in range(reps):
        with torch.cuda.stream(st):
            a.record(st)
            A_dev.copy_(A_host, non_blocking=True)
            b.record(st)
        torch.cuda.synchronize()
        h2d.append(A_host.numel() * A_host.element_size() / (a.elapsed_time(b) * 1e-3) / 1e9)
        with torch.cuda.stream(st):
            a.record(st)
            theta_host.copy_(theta_dev, non_blocking=True)
            b.record(st)
        torch.cuda.synchronize()
        d2h.append(theta_host.numel() * theta_host.element_size() / (a.elapsed_time(b) * 1e-3) / 1e9)
    return max(h2d), max(d2h)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def make_input(cfg):
    return W.dense_lowrank_skewed(cfg["n"], cfg["d"], cfg["rank"], seed=cfg["data_seed"])


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_step(A, cfg):
    from oracle import estimator as E
    return E.estimate(A.astype(np.float64, copy=False), cfg["s"], cfg["m"], cfg["k"], cfg["tau"], cfg["seed"])


def run_reference(args, cfg):
    """The FP64 CPU oracle as it stands, on row-prefix samples of the workload."""
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    A = make_input(cfg)
    budget = 200.0 / max(1, args.steps + args.warmup)            # seconds of CPU work per step
    n_s = cfg["n"] if budget >= 20 else max(65536, int(cfg["n"] * budget / 20.0))
    sample = A[:n_s]
    for _ in range(args.warmup):
        oracle_step(sample, cfg)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(sample, cfg)
    dt = (time.perf_counter() - t0) / args.steps
    value = n_s / dt
    desc = f"row prefix of {n_s} of {cfg['n']} rows per step, same s, m, k (fixed costs included)"
    out = {"metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "n": cfg["n"], "d": cfg["d"], "s": cfg["s"], "m": cfg["m"],
                      "k": cfg["k"], "parallelism": "replicas"},
           "cpu_baseline": {"value": value, "unit": "rows/s", "cores": cpu_threads(), "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def qr_flops(m, d, r):
    """FP64 flops of the pivoted Householder QR that stops at rank r (norm recompute included)."""
    f = 0.0
    for j in range(r):
        rows, cols = m - j, d - j - 1
        f += 6.0 * rows * cols + 2.0 * rows
    return f


def run_stage(a):
    """One stage of the path on a seeded synthetic case, a few times, for a profiler (ncu -k/-s/-c):
    prints the CUDA-event time of the last repetition. Inputs come from the workloads module; every
    stage runs through the C ABI as lev_estimate_* runs it."""
    import torch
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
        # shaped as the estimator's factor: rank nonzero rows (the selected columns) and, when
        # rank < k, its first rank columns (the reduced form of lev_omega_factor)
        rs = np.random.default_rng(a.seed)
        M = rs.standard_normal((a.d, a.k)) / np.sqrt(a.d)
        r = min(a.rank, a.d)
        M[rs.permutation(a.d)[r:], :] = 0.0
        if r < a.k:
            M[:, r:] = 0.0
        Mf = torch.from_numpy(M.astype(np.float32)).cuda()
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sketch-prec", default="bf16x3")
    ap.add_argument("--final-prec", default="bf16x3")
    ap.add_argument("--forms", default="fp32,tf32,bf16,bf16x3",
                    help="whole-path forms timed and checked: fp32 = FP32 SIMT sketch and final pass; "
                         "tf32 / bf16 / bf16x3 = split-BF16 tensor-core sketch with that final-pass form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-exact", action="store_true", help="skip the Alg. 7 (LS-HRN-exact) measurement")
    ap.add_argument("--no-extras", action="store_true", help="skip the rank-rule and least-squares measurements")
    ap.add_argument("--no-csr", action="store_true", help="skip the CSR 8e6 x 1024 measurement")
    ap.add_argument("--no-csr-large", action="store_true", help="skip the CSR 8e7 x 1024 (~1e9 nnz) workload")
    ap.add_argument("--streams", type=int, default=6,
                    help="batches in flight: step i runs on stream i mod S with its own handle, so one batch's "
                         "latency-bound pivoted Cholesky overlaps another batch's HBM- and tensor-bound kernels")
    # profiling mode: one stage on a synthetic case (see run_stage)
    ap.add_argument("--stage", choices=["final", "rrqr", "sketch", "backward", "lsqr", "svd", "exact_csr",
                                        "estimate_csr"], help="run one stage a few times for a profiler")
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
    args = ap.parse_args()
    if args.stage:
        run_stage(args)
        return
    args.warmup = max(3, args.warmup)
    cfg = W.CONFIGS[WORKLOAD]
    if args.impl == "reference":
        run_reference(args, cfg)
        return

    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    import paper_2105_11004_gb300 as L

    placement = gpu_numa_placement(local)            # before any pinned host buffer exists
    large = {}
    gen_thread = None
    n, d = cfg["n"], cfg["d"]
    A_np = make_input(cfg)
    A_host = torch.from_numpy(A_np).pin_memory()
    A = A_host.cuda()
    h = L.Handle(local)

    def params(final_prec):
        return L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"],
                             sketch_prec=args.sketch_prec, final_prec=final_prec)

    p = params(args.final_prec)
    theta = torch.empty(n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    # cacheable setup (the handle keeps G, the bucket permutation and Omega per seed and sizes):
    # lev_prepare timed with a seed the handle has not seen, after a first call has sized the buffers
    L.lev_prepare(h, n, d, p)
    torch.cuda.synchronize()
    q = L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"] + 1000,
                      sketch_prec=args.sketch_prec)
    a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_.record(stream)
    L.lev_prepare(h, n, d, q)
    b_.record(stream)
    torch.cuda.synchronize()
    setup = {"ms": a_.elapsed_time(b_)}
    setup["what"] = (f"G ({cfg['m']} x {cfg['s']}, BF16 hi + lo pair of the FP32 draws), the CountSketch bucket "
                     f"permutation ({n} rows) and Omega ({d} x {cfg['k']}) for a new seed (lev_prepare)")
    # kernels of one lev_estimate_dense step with the bucket permutation, G and Omega cached:
    # CountSketch (FP32 B, or for the BF16 forms the Gaussian stage's operand itself), the Gaussian
    # stage (split-K SGEMM or tcgen05 GEMM) and its reduction; Gram + reduce + pivoted Cholesky (one
    # cluster at d <= 256) + the FP64 conversion of R + two assembly kernels; the coefficient split
    # and the solve of the right factor; the final pass (tensor-core forms: plus its width and
    # operand packing kernels)
    kernels_per_step = (3 + (1 if args.sketch_prec == "tf32" else 0) + 6 + 2
                        + (1 if args.final_prec == "fp32" else 3))

    rank_found = L.lev_estimate_dense(h, A, p, theta)          # also generates and caches G
    # S batches in flight: handle i and stream i take steps i, i + S, ... (each handle holds its own
    # scratch and caches; every step is the whole path on the whole batch)
    S = max(1, args.streams)
    hs = [h] + [L.Handle(local) for _ in range(S - 1)]
    sts = [torch.cuda.Stream() for _ in range(S)]
    ths = [theta] + [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(S - 1)]
    for i in range(S):
        L.lev_estimate_dense(hs[i], A, p, ths[i], stream=sts[i])   # caches of every handle
    torch.cuda.synchronize()
    for t in range(args.warmup):
        L.lev_estimate_dense(hs[t % S], A, p, ths[t % S], want_rank=False, stream=sts[t % S])
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    e0.record(stream)
    for st_ in sts:
        st_.wait_stream(stream)
    for t in range(args.steps):
        L.lev_estimate_dense(hs[t % S], A, p, ths[t % S], want_rank=False, stream=sts[t % S])
    for st_ in sts:
        stream.wait_stream(st_)
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    barrier(world)
    ms = allmax(world, e0.elapsed_time(e1) / args.steps)
    clocks = sampler.summary(t_wall0, t_wall1)
    sampler.stop()
    same_theta = all(torch.equal(ths[0], t_) for t_ in ths[1:])

    e2e_out = None
    if not args.no_e2e:
        # end to end through the public API with pinned host A and theta: every step copies A
        # (1.02 GB) host -> device and theta (4 MB) back. LEV_HOST_ASYNC lets the call return once
        # its work is enqueued, so the handle's copy stream moves step i+1's A while the kernels
        # of step i run; the loop ends with a synchronisation and the copied theta is checked.
        pa = L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"],
                           sketch_prec=args.sketch_prec, final_prec=args.final_prec, host_async=True)
        theta_host = torch.empty(n, dtype=torch.float32).pin_memory()
        theta_dev = torch.empty(n, dtype=torch.float32, device="cuda")
        L.lev_estimate_dense(h, A, pa, theta_dev)
        for _ in range(2):
            L.lev_estimate_dense(h, A_host, pa, theta_host, want_rank=False)
        torch.cuda.synchronize()
        barrier(world)
        ke = max(5, min(args.steps, 20))
        # three repetitions of the ke-step loop; the line reports their median and lists all three
        reps_e2e, enq = [], []
        for _ in range(3):
            t0 = time.perf_counter()
            for _ in range(ke):
                L.lev_estimate_dense(h, A_host, pa, theta_host, want_rank=False)
            t_enq = time.perf_counter()
            torch.cuda.synchronize()
            reps_e2e.append(allmax(world, (time.perf_counter() - t0) / ke))
            enq.append((t_enq - t0) / ke)
        te = float(np.median(reps_e2e))
        same = bool(np.array_equal(theta_host.numpy(), theta_dev.cpu().numpy()))
        h2d_gbs, d2h_gbs = host_link(A_host, torch.empty_like(A), theta_host, theta_dev)
        e2e_out = {"value": n * world / te, "unit": "rows/s", "h2d_bytes_per_step": n * d * 4,
                   "d2h_bytes_per_step": n * 4, "ms_per_step": te * 1e3, "steps": ke,
                   "h2d_gbs_measured": h2d_gbs, "d2h_gbs_measured": d2h_gbs,
                   "h2d_floor_ms": n * d * 4 / (h2d_gbs * 1e9) * 1e3,
                   "floor_source": "pinned 1.02 GB host -> device copy timed by CUDA events in this run",
                   "api": "lev_estimate_dense, pinned host A and theta, LEV_HOST_ASYNC (copy of step i+1 "
                          "overlaps the kernels of step i; one synchronisation after the loop; median of "
                          "three loops)",
                   "theta_equals_device_path": same,
                   "repetitions_ms_per_step": [x * 1e3 for x in reps_e2e],
                   "host_enqueue_ms_per_step": [x * 1e3 for x in enq]}

    # the ~1e9-nonzero CSR workload takes about a minute to generate on the host: start it now, in a
    # thread, so that it overlaps the GPU work of the other sections (after the headline step and the
    # end-to-end copies, which it would disturb)
    if not args.no_csr and not args.no_csr_large:
        def _gen_large():
            c = W.CONFIGS["csr_8e7x1024_rank1014"]
            t0 = time.perf_counter()
            large["C"] = W.csr_dup_columns(c["n"], c["d"], seed=c["data_seed"])
            large["gen_s"] = time.perf_counter() - t0
        gen_thread = threading.Thread(target=_gen_large, daemon=True)
        gen_thread.start()

    def time_steps(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    reps = max(3, min(args.steps, 20))
    # every final-pass form: whole-step time and theta~ for the accuracy check
    forms = {}
    form_theta = {}
    for f in [x for x in args.forms.split(",") if x]:
        pf = L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"],
                           sketch_prec="fp32" if f == "fp32" else "bf16x3", final_prec=f)
        tf = torch.empty(n, dtype=torch.float32, device="cuda")
        L.lev_estimate_dense(h, A, pf, tf)
        form_theta[f] = tf.cpu().numpy()
        t_ms = time_steps(lambda: L.lev_estimate_dense(h, A, pf, tf, want_rank=False), reps)
        forms[f] = {"ms_per_step": t_ms, "rows_per_s": n / (t_ms * 1e-3),
                    "sketch_prec": "fp32" if f == "fp32" else "bf16x3", "final_prec": f}

    # per-stage times (same inputs, same stream) for the rooflines
    At = torch.empty((cfg["m"], d), dtype=torch.float32, device="cuda")
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    R = torch.empty((d, d), dtype=torch.float64, device="cuda")
    Mf = torch.empty((d, cfg["k"]), dtype=torch.float32, device="cuda")
    L.lev_sketch_dense(h, A, p, At)
    r = L.lev_rrqr(h, At, cfg["tau"], perm, R)
    d_rank = torch.tensor([r], dtype=torch.int64, device="cuda")
    L.lev_omega_factor(h, R, perm, d_rank, d, cfg["k"], cfg["seed"], L.LEV_OMEGA_REDUCED, Mf)
    stages = {
        "sketch": time_steps(lambda: L.lev_sketch_dense(h, A, p, At), reps),
        "rrqr": time_steps(lambda: lib_rrqr_nosync(L, h, At, cfg["tau"], perm, R), reps),
        "omega": time_steps(lambda: L.lev_omega_factor(h, R, perm, d_rank, d, cfg["k"], cfg["seed"],
                                                       L.LEV_OMEGA_REDUCED, Mf), reps),
    }
    final_call_ms = {f: time_steps(lambda f=f: L.lev_final_dense(h, A, Mf, f, theta), reps)
                     for f in sorted(set(list(forms) + [args.final_prec]))}
    stages["final"] = final_call_ms[args.final_prec]
    # the main kernel of each tensor-core final pass alone (events the library records around its
    # launch, after the packing of Mfull's operand image); the FP32 SIMT pass is one kernel
    L.lev_set_timing(h, True)
    final_ms = {}
    for f in final_call_ms:
        if f == "fp32":
            final_ms[f] = final_call_ms[f]
            continue
        ks = []
        for _ in range(reps):
            L.lev_final_dense(h, A, Mf, f, theta)
            ks.append(L.lev_final_timing(h))
        final_ms[f] = float(np.median(ks))
    L.lev_set_timing(h, False)
    # MMA width of the tensor-core pass: Mfull's columns up to its last nonzero one, rounded up to 16
    nz_cols = np.nonzero(np.any(Mf.cpu().numpy() != 0, axis=0))[0]
    mma_n = max(16, -(-(int(nz_cols[-1]) + 1 if nz_cols.size else 0) // 16) * 16)
    # the two kernels of the QR stage, from CUDA events the library records on the launching
    # stream around them (lev_set_timing): the Gram product and the grid pivoted Cholesky
    L.lev_set_timing(h, True)
    gram_ms, chol_ms = [], []
    for _ in range(reps):
        L.lev_rrqr(h, At, cfg["tau"], perm, R)
        g_ms, f_ms = L.lev_rrqr_timing(h)
        gram_ms.append(g_ms)
        chol_ms.append(f_ms)
    L.lev_set_timing(h, False)
    # the pivoted Cholesky runs on one thread-block cluster up to d = 256, on a cooperative grid above
    pchol_name = "k_pchol_cluster" if d <= 256 else "k_pchol_grid"
    kernel_ms = {"k_final_tc": final_ms[args.final_prec], pchol_name: float(np.median(chol_ms)),
                 "k_gram_dot2+reduce": float(np.median(gram_ms))}

    peaks, peak_src = load_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    fp32_peak = 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    final_bytes = n * d * 4 + n * 4 + d * cfg["k"] * 4
    final_flops = 2.0 * n * r * cfg["k"]

    def final_roof(f):
        t = final_ms[f] * 1e-3
        if f == "fp32":
            roof = {"kernel": "k_final_dense_fp32", "bound": "alu", "achieved": final_flops / t / 1e12,
                    "peak": fp32_peak, "unit": "TFLOP/s",
                    "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock",
                    "algorithmic": final_flops}
        else:
            roof = {"kernel": f"k_final_tc<{f}>", "bound": "hbm", "achieved": final_bytes / t / 1e9,
                    "peak": hbm_peak, "unit": "GB/s", "peak_source": f"hbm_gbs ({peak_src})",
                    "algorithmic": final_bytes}
            # the tensor pipe: executed MMA flops per form (K = d rounded up to the 64-column K
            # block, N = mma_n; the split form runs three products hi*hi + lo*hi + hi*lo)
            mult = {"bf16": 1, "tf32": 1, "bf16x3": 3}[f]
            peak_tc = float(peaks.get("bf16_tflops", 1900.0)) * (0.5 if f == "tf32" else 1.0)
            exec_flops = mult * 2.0 * n * mma_n * (-(-d // 64) * 64)
            roof["tensor"] = {"achieved": exec_flops / t / 1e12, "peak": peak_tc, "unit": "TFLOP/s",
                              "frac": exec_flops / t / 1e12 / peak_tc, "executed_flops": exec_flops,
                              "peak_source": "bf16_tflops burst (measured)"
                              + (" x 1/2 (TF32 nominal ratio)" if f == "tf32" else "")}
        roof["frac"] = roof["achieved"] / roof["peak"]
        # DRAM bytes per launch from the ncu capture of this kernel (split BF16) on 262,144 x 256 with
        # an Mfull of 208 nonzero columns, scaled by rows: read 268,712,704 + write 3,499,264 bytes
        roof["traffic"] = ((268712704 + 3499264) * n / 262144
                           if (f == "bf16x3" and d == 256 and mma_n == 208) else None)
        roof["ms"] = final_ms[f]
        roof["call_ms"] = final_call_ms[f]
        roof["mma_n"] = mma_n if f != "fp32" else None
        return roof

    rooflines = {"final": final_roof(args.final_prec)}
    sk_bytes = n * d * 4 + cfg["s"] * d * 4
    sk_kernels = {"bf16x3": "k_countsketch_dense_op (writes the operand) + k_gauss_tc + k_gauss_reduce",
                  "bf16": "k_countsketch_dense_op (writes the operand) + k_gauss_tc + k_gauss_reduce",
                  "tf32": "k_countsketch_dense_v4 + k_transpose_operand + k_gauss_tc + k_gauss_reduce",
                  "fp32": "k_countsketch_dense_v4 + split-K SGEMM + reduction"}[args.sketch_prec]
    rooflines["sketch"] = {"kernels": sk_kernels, "bound": "mixed",
                           "ms": stages["sketch"],
                           "countsketch_bytes": sk_bytes, "gemm_flops": 2.0 * cfg["m"] * cfg["s"] * d}
    qf = qr_flops(cfg["m"], d, r)
    fp64_peak = 1.19   # TFLOP/s, FP64 FMA rate measured on this GB300 (dependent-chain probe)
    chol_flops = 2.0 * sum((d - j) ** 2 for j in range(r))          # rank-1 updates of the trailing block
    rooflines["rrqr"] = {"kernels": f"k_gram_dot2 + k_gram_reduce, {pchol_name}", "ms": stages["rrqr"],
                         "gram_ms": kernel_ms["k_gram_dot2+reduce"], "pchol_ms": kernel_ms[pchol_name],
                         "pchol_us_per_step": kernel_ms[pchol_name] * 1e3 / max(1, r),
                         "householder_equivalent_fp64_flops": qf,
                         "note": f"{r} sequential pivot steps; one exchange of the pivot column per step "
                                 f"({'shared memory across the cluster' if d <= 256 else 'L2'})"}
    rooflines["pchol"] = {"kernel": pchol_name, "bound": "alu",
                          "achieved": chol_flops / (kernel_ms[pchol_name] * 1e-3) / 1e12, "peak": fp64_peak,
                          "unit": "TFLOP/s", "peak_source": "FP64 FMA rate measured on this GB300 (1.19 TFLOP/s)",
                          "algorithmic": chol_flops, "traffic": None, "ms": kernel_ms[pchol_name],
                          "note": "latency-bound: each pivot step waits for the pivot column from the CTA that "
                                  "owns it (a remote shared-memory hop of about 250 ns in the cluster form, an L2 "
                                  "round trip in the grid form) and a chain of dependent double-float (FP32 pair) "
                                  "operations; achieved is counted in FP64-equivalent flops, whose whole count "
                                  "would take ~9 us at the FP64 rate"}
    rooflines["pchol"]["frac"] = rooflines["pchol"]["achieved"] / fp64_peak
    dominant_kernel = max(kernel_ms, key=kernel_ms.get)
    dominant = max(stages, key=stages.get)
    # the roofline line is the dominant kernel's; the final pass (the kernel that moves the
    # workload's bytes) stays beside it
    roof = rooflines["pchol"] if dominant_kernel == pchol_name else rooflines["final"]

    out = {"metric": METRIC, "value": n * world / (ms * 1e-3), "unit": "rows/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": n, "d": d, "rank": cfg["rank"], "s": cfg["s"], "m": cfg["m"],
                      "k": cfg["k"], "tau": cfg["tau"], "sketch_prec": args.sketch_prec,
                      "final_prec": args.final_prec, "parallelism": "replicas" if world > 1 else "single",
                      "l2": "inputs larger than L2 (A is 1.02 GB), no flush",
                      "cached": "per handle: G (m x s) per seed, the bucket permutation per (seed, n, s), Omega "
                                "per (seed, d, k); every stage of the path runs every step",
                      "batches_in_flight": S},
           "rank_found": rank_found, "stages_ms": stages, "final_ms_by_form": final_ms, "forms": forms,
           "ms_per_step_one_batch_in_flight": forms.get(args.final_prec, {}).get("ms_per_step"),
           "theta_equal_across_streams": same_theta,
           "setup_ms": setup, "host_placement": placement,
           "step_hbm": {"algorithmic_bytes": 2 * n * d * 4 + cfg["s"] * d * 4 + n * 4,
                        "gbs_one_batch": None, "gbs_batches_in_flight": (2 * n * d * 4 + cfg["s"] * d * 4 + n * 4)
                        / (ms * 1e-3) / 1e9, "note": "A read twice (CountSketch, final pass), B written, theta written"},
           "roofline": roof, "dominant_stage": dominant, "dominant_kernel": dominant_kernel,
           "kernel_ms": kernel_ms, "rooflines": rooflines,
           "roofline_final_pass": rooflines["final"],
           "clocks": clocks, "gpu_launches": kernels_per_step * args.steps}
    one = out["ms_per_step_one_batch_in_flight"]
    if one:
        out["step_hbm"]["gbs_one_batch"] = out["step_hbm"]["algorithmic_bytes"] / (one * 1e-3) / 1e9

    # Alg. 7 (LS-HRN-exact) on the same batch: the sketch's QR selects K, the FP64 Gram matrix of A
    # (2.1e10 FMA at n = 1e6, d = 256) gives B = A_K^T A_K, then its Cholesky and the final pass
    if not args.no_exact:
        pe = L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"],
                           sketch_prec=args.sketch_prec, final_prec=args.final_prec)
        th_e = torch.empty(n, dtype=torch.float32, device="cuda")
        r_e = L.lev_exact_dense(h, A, pe, th_e)
        ex_ms = time_steps(lambda: L.lev_exact_dense(h, A, pe, th_e), 3)
        # the Gram product of A alone: the QR of A itself runs it (timing marks of the library)
        L.lev_set_timing(h, True)
        pa = torch.empty(d, dtype=torch.int32, device="cuda")
        Ra = torch.empty((d, d), dtype=torch.float64, device="cuda")
        L.lev_rrqr(h, A, cfg["tau"], pa, Ra)
        g_ms, _ = L.lev_rrqr_timing(h)
        L.lev_set_timing(h, False)
        gram_fma = n * d * (d + 32) / 2.0            # upper 32 x 32 tiles, diagonal tiles in full
        out["exact"] = {"algorithm": "Alg. 7 (LS-HRN-exact), lev_exact_dense", "rank": r_e, "ms_per_call": ex_ms,
                        "rows_per_s": n / (ex_ms * 1e-3), "gram_ms": g_ms,
                        "gram_fp64_equivalent_tflops": 2.0 * gram_fma / (g_ms * 1e-3) / 1e12,
                        "fp64_peak_tflops": fp64_peak,
                        "gram_note": "compensated FP32 sums (exact products, TwoSum blocks of 64 rows, FP64 outer sum)",
                        "sketch_prec": args.sketch_prec, "final_prec": args.final_prec}

    # rank rules on the same batch's sketch (lev_rrqr_select): the diagonal test, the singular values
    # of the sketch (Alg. 11 step 3), strong-RRQR swaps (Alg. 2)
    if not args.no_extras:
        ps = L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"],
                           sketch_prec=args.sketch_prec)
        At_r = torch.empty((cfg["m"], d), dtype=torch.float32, device="cuda")
        L.lev_sketch_dense(h, A, ps, At_r)
        pr = torch.empty(d, dtype=torch.int32, device="cuda")
        Rr = torch.empty((d, d), dtype=torch.float64, device="cuda")
        rules = {}
        for name, kw in [("diag", {}), ("svd", dict(rank_svd=True)), ("srrqr_phi2", dict(srrqr_phi=2.0)),
                         ("svd_srrqr_phi1.05", dict(rank_svd=True, srrqr_phi=1.05))]:
            pk = L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"], **kw)
            rk, sw = L.lev_rrqr_select(h, At_r, pk, pr, Rr)
            rules[name] = {"rank": rk, "swaps": sw,
                           "ms": time_steps(lambda: L.lev_rrqr_select(h, At_r, pk, pr, Rr), 3)}
        out["rank_rules"] = {"sketch": f"{cfg['m']} x {d}", "rules": rules}
        out["lstsq"] = lstsq_timing(L, h, n, d, time_steps)

    # backward workload: dense 200,000 x 64, s = 16,384, m = 256, k = 128; forward = the four stages
    if not args.no_backward:
        out["backward"] = backward_timing(L, h, reps)

    if e2e_out is not None:
        out["e2e"] = e2e_out
    if not args.no_csr:
        out["csr"] = {"csr_8e6x1024": csr_timing(L, h, "csr_8e6x1024", reps)}
        if gen_thread is not None:
            t0 = time.perf_counter()
            gen_thread.join()
            wait_s = time.perf_counter() - t0
            out["csr"]["csr_8e7x1024_rank1014"] = csr_large_timing(L, h, "csr_8e7x1024_rank1014", 3, large)
            out["csr"]["csr_8e7x1024_rank1014"]["generation_wait_s"] = wait_s
            large.clear()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        runs = []
        for _ in range(3):
            t0 = time.perf_counter()
            est = oracle_step(A_np, cfg)
            runs.append(time.perf_counter() - t0)
        dt = float(np.median(runs))
        one = single_thread_oracle(cfg, 262144)
        out["cpu_baseline"] = {"value": n / dt, "unit": "rows/s", "cores": cpu_threads(), "kind": "oracle",
                               "sample": "the FP64 oracle on the full workload, median of 3 runs", "seconds": runs,
                               "cpu_model": cpu_model(), "single_thread": one}
        out["oracle_rank"] = est.rank
        for f, th in form_theta.items():
            rel = np.abs(th.astype(np.float64) - est.theta) / est.theta
            forms[f]["max_rel_err_vs_oracle"] = float(rel.max())
            forms[f]["p99_rel_err_vs_oracle"] = float(np.quantile(rel, 0.99))
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def csr_timing(L, h, name, reps):
    """Whole estimate on a CSR workload (split-BF16 Gaussian stage, FP32 CSR final pass), with stages."""
    import torch
    cfg = W.CONFIGS[name]
    n, d = cfg["n"], cfg["d"]
    t0 = time.perf_counter()
    C = W.csr_uniform(n, d, seed=cfg["data_seed"]) if name == "csr_8e6x1024" else \
        W.csr_dup_columns(n, d, seed=cfg["data_seed"])
    gen_s = time.perf_counter() - t0
    rp = torch.from_numpy(C.row_ptr).cuda()
    cl = torch.from_numpy(C.col).cuda()
    vl = torch.from_numpy(C.val).cuda()
    p = L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"], sketch_prec="bf16x3")
    theta = torch.empty(n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    r = L.lev_estimate_csr(h, rp, cl, vl, n, d, p, theta)

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    ms = timed(lambda: L.lev_estimate_csr(h, rp, cl, vl, n, d, p, theta, want_rank=False), reps)
    # cacheable setup for a new seed: G (4096 x 262144 as the BF16 pair), bucket permutation, Omega
    setup_ms = timed(lambda: L.lev_prepare(h, n, d, L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"],
                                                                   seed=int(time.time_ns() % 10**9),
                                                                   sketch_prec="bf16x3")), 1)
    L.lev_prepare(h, n, d, p)
    At = torch.empty((cfg["m"], d), dtype=torch.float32, device="cuda")
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    R = torch.empty((d, d), dtype=torch.float64, device="cuda")
    Mf = torch.empty((d, cfg["k"]), dtype=torch.float32, device="cuda")
    L.lev_sketch_csr(h, rp, cl, vl, n, d, p, At)
    L.lev_rrqr(h, At, cfg["tau"], perm, R)
    d_rank = torch.tensor([r], dtype=torch.int64, device="cuda")
    L.lev_omega_factor(h, R, perm, d_rank, d, cfg["k"], cfg["seed"], L.LEV_OMEGA_REDUCED, Mf)
    stages = {"sketch": timed(lambda: L.lev_sketch_csr(h, rp, cl, vl, n, d, p, At), reps),
              "rrqr": timed(lambda: lib_rrqr_nosync(L, h, At, cfg["tau"], perm, R), reps),
              "omega": timed(lambda: L.lev_omega_factor(h, R, perm, d_rank, d, cfg["k"], cfg["seed"],
                                                        L.LEV_OMEGA_REDUCED, Mf), reps),
              "final": timed(lambda: L.lev_final_csr(h, rp, cl, vl, n, d, Mf, "fp32", theta), reps)}
    csr_bytes = C.nnz * 8 + (n + 1) * 8
    out = {"n": n, "d": d, "nnz": C.nnz, "rank": r, "ms_per_step": ms, "rows_per_s": n / (ms * 1e-3),
           "csr_gbs_two_passes": 2 * csr_bytes / (ms * 1e-3) / 1e9, "stages_ms": stages, "setup_ms": setup_ms,
           "sketch_prec": "bf16x3", "final_prec": "fp32", "generation_s": gen_s}
    # the same estimate with an SRHT after the CountSketch (Sec. 4.1): t from the quoted SRHT
    # theorem, 4 (sqrt(d) + sqrt(ln(s d)))^2 ln d, rounded up to a multiple of 64
    t = int(np.ceil(4 * (np.sqrt(d) + np.sqrt(np.log(cfg["s"] * d))) ** 2 * np.log(d) / 64.0) * 64)
    ps = L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"], sketch_prec="bf16x3",
                       srht_t=t)
    r_s = L.lev_estimate_csr(h, rp, cl, vl, n, d, ps, theta)
    ms_s = timed(lambda: L.lev_estimate_csr(h, rp, cl, vl, n, d, ps, theta, want_rank=False), reps)
    sk_s = timed(lambda: L.lev_sketch_csr(h, rp, cl, vl, n, d, ps, At), reps)
    out["srht"] = {"t": t, "rank": r_s, "ms_per_step": ms_s, "rows_per_s": n / (ms_s * 1e-3), "sketch_ms": sk_s,
                   "gaussian_stage_flops": 2.0 * cfg["m"] * t * d, "note": "A~ = G (F (S A)), G m x t"}
    # Alg. 11 and LSQR on the same matrix with b ~ N(0, 1): min ||A x - b|| for CSR A
    b = torch.from_numpy(np.random.default_rng(0).standard_normal(n).astype(np.float32)).cuda()
    pn = L.make_params(s=cfg["s"], m=cfg["m"], k=8, tau=1e-10, seed=cfg["seed"], sketch_prec="bf16x3")
    Np = torch.empty((d, d), dtype=torch.float64, device="cuda")
    kp = L.lev_precondition_csr(h, rp, cl, vl, n, d, pn, Np)
    pre_ms = timed(lambda: L.lev_precondition_csr(h, rp, cl, vl, n, d, pn, Np), 1)
    xs = torch.zeros(d, dtype=torch.float64, device="cuda")
    its, rns = L.lev_lsqr_csr(h, rp, cl, vl, n, d, Np, kp, b, xs)
    ls_ms = timed(lambda: L.lev_lsqr_csr(h, rp, cl, vl, n, d, Np, kp, b, xs), 2)
    out["lstsq"] = {"rank": kp, "precondition_ms": pre_ms, "iterations": its, "lsqr_ms": ls_ms,
                    "csr_gbs_per_pass": (its + 1) * (csr_bytes + 8 * n) / (ls_ms * 1e-3) / 1e9}
    # Alg. 7 (LS-HRN-exact) on the same matrix: B = A_K^T A_K from the rows' outer products
    # (Lemma 8, Sec. 5.1, FP64), its forced-pivot Cholesky, theta = ||A_K R^{-1}||^2 (k = d)
    r_e = L.lev_exact_csr(h, rp, cl, vl, n, d, p, theta)
    ms_e = timed(lambda: L.lev_exact_csr(h, rp, cl, vl, n, d, p, theta), max(1, reps // 2))
    lens = np.diff(C.row_ptr).astype(np.float64)
    out["exact"] = {"algorithm": "Alg. 7 (LS-HRN-exact), lev_exact_csr", "rank": r_e, "ms_per_call": ms_e,
                    "rows_per_s": n / (ms_e * 1e-3), "gram_pairs": float(np.sum(lens * (lens + 1) / 2)),
                    "note": "three host synchronisations per call (after each factorisation and after counting the long rows)"}
    return out


def csr_large_timing(L, h, name, reps, pre):
    """The whole estimate on the CSR 8e7 x 1024 workload (~1e9 nonzeros; split-BF16 Gaussian stage,
    FP32 CSR final pass), generated on the host beforehand (pre["C"]): setup, step time, stages, rank."""
    import torch
    cfg = W.CONFIGS[name]
    n, d = cfg["n"], cfg["d"]
    C = pre.pop("C")
    gen_s = pre.get("gen_s")
    rp, cl, vl = (torch.from_numpy(x).cuda() for x in (C.row_ptr, C.col, C.val))
    del C
    nnz = cl.numel()
    p = L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"], sketch_prec="bf16x3")
    theta = torch.empty(n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    setup_ms = timed(lambda: L.lev_prepare(h, n, d, L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"],
                                                                   tau=cfg["tau"], seed=int(time.time_ns() % 10**9),
                                                                   sketch_prec="bf16x3")), 1)
    r = L.lev_estimate_csr(h, rp, cl, vl, n, d, p, theta)
    ms = timed(lambda: L.lev_estimate_csr(h, rp, cl, vl, n, d, p, theta, want_rank=False), reps)
    At = torch.empty((cfg["m"], d), dtype=torch.float32, device="cuda")
    perm = torch.empty(d, dtype=torch.int32, device="cuda")
    R = torch.empty((d, d), dtype=torch.float64, device="cuda")
    Mf = torch.empty((d, cfg["k"]), dtype=torch.float32, device="cuda")
    L.lev_sketch_csr(h, rp, cl, vl, n, d, p, At)
    L.lev_rrqr(h, At, cfg["tau"], perm, R)
    d_rank = torch.tensor([r], dtype=torch.int64, device="cuda")
    L.lev_omega_factor(h, R, perm, d_rank, d, cfg["k"], cfg["seed"], L.LEV_OMEGA_REDUCED, Mf)
    stages = {"sketch": timed(lambda: L.lev_sketch_csr(h, rp, cl, vl, n, d, p, At), reps),
              "rrqr": timed(lambda: lib_rrqr_nosync(L, h, At, cfg["tau"], perm, R), reps),
              "omega": timed(lambda: L.lev_omega_factor(h, R, perm, d_rank, d, cfg["k"], cfg["seed"],
                                                        L.LEV_OMEGA_REDUCED, Mf), reps),
              "final": timed(lambda: L.lev_final_csr(h, rp, cl, vl, n, d, Mf, "fp32", theta), reps)}
    csr_bytes = nnz * 8 + (n + 1) * 8
    out = {"n": n, "d": d, "nnz": nnz, "rank": r, "ms_per_step": ms, "rows_per_s": n / (ms * 1e-3),
           "csr_gbs_two_passes": 2 * csr_bytes / (ms * 1e-3) / 1e9, "stages_ms": stages, "setup_ms": setup_ms,
           "sketch_prec": "bf16x3", "final_prec": "fp32", "generation_s": gen_s,
           "note": "row_ptr checked once per call; setup = G, bucket permutation and Omega for a new seed"}
    del rp, cl, vl
    torch.cuda.empty_cache()
    return out


def single_thread_oracle(cfg, rows):
    """The FP64 oracle on a `rows`-row matrix of the dense workload's recipe (same rank, row scaling,
    seed, s, m, k) in a child process whose BLAS and OpenMP pools have one thread: rows/s on one core,
    a bounded sample (the fixed cost of generating G is included)."""
    code = ("import os, sys, time\n"
            "sys.path.insert(0, %r)\n"
            "import numpy as np, workloads as W\n"
            "from oracle import estimator as E\n"
            "A = W.dense_lowrank_skewed(%d, %d, %d, seed=%d)[:%d].astype(np.float64)\n"
            "t0 = time.perf_counter(); E.estimate(A, %d, %d, %d, %r, %d); print(time.perf_counter() - t0)\n"
            % (ROOT, rows, cfg["d"], cfg["rank"], cfg["data_seed"], rows, cfg["s"], cfg["m"], cfg["k"], cfg["tau"],
               cfg["seed"]))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
        sec = float(r.stdout.strip().splitlines()[-1])
        return {"value": rows / sec, "unit": "rows/s", "cores": 1, "seconds": sec,
                "sample": f"a {rows}-row matrix of the dense workload's recipe, same s, m, k, one thread"}
    except Exception as e:
        return {"error": str(e)[:200]}


def lstsq_timing(L, h, n, d, time_steps):
    """Alg. 11 (CountGauss preconditioner) and LSQR on A N for a dense n x d least-squares problem:
    A with lognormal row scales (the batch's distribution at full rank), b ~ N(0, 1)."""
    import torch
    rs = np.random.default_rng(0)
    A = torch.from_numpy(W.dense_lowrank_skewed(n, d, d, seed=1)).cuda()
    b = torch.from_numpy(rs.standard_normal(n).astype(np.float32)).cuda()
    p = L.make_params(s=65536, m=4 * d, k=8, tau=1e-10, seed=3, sketch_prec="bf16x3")
    N = torch.empty((d, d), dtype=torch.float64, device="cuda")
    k = L.lev_precondition_dense(h, A, p, N)
    pre_ms = time_steps(lambda: L.lev_precondition_dense(h, A, p, N), 3)
    x = torch.zeros(d, dtype=torch.float64, device="cuda")
    it, rn = L.lev_lsqr_dense(h, A, N, k, b, x, max_iter=200, atol=1e-6, btol=1e-6)
    ls_ms = time_steps(lambda: L.lev_lsqr_dense(h, A, N, k, b, x, max_iter=200, atol=1e-6, btol=1e-6), 5)
    passes = it + 1
    pass_bytes = n * d * 4 + 2 * n * 4                 # A once, u read and written
    return {"problem": f"dense {n} x {d}, lognormal row scales, b ~ N(0,1)", "rank": k, "iterations": it,
            "precondition_ms": pre_ms, "lsqr_ms": ls_ms, "residual": rn,
            "lsqr_gbs_per_pass": passes * pass_bytes / (ls_ms * 1e-3) / 1e9,
            "note": "one fused pass over A per iteration (A N v and A^T u' together); GB/s counts the whole "
                    "solve including the small FP64 steps and one host check per 16 iterations"}


def backward_timing(L, h, reps):
    """Forward (sketch, rrqr, omega factor, final pass) and backward times on the backward workload."""
    import torch
    cfg = W.CONFIGS["dense_2e5x64_backward"]
    A = torch.from_numpy(W.dense_heavy_rows(cfg["n"], cfg["d"], seed=cfg["data_seed"])).cuda()
    w = torch.from_numpy(W.uniform_weights(cfg["n"], seed=cfg["weight_seed"])).cuda()
    p = L.make_params(s=cfg["s"], m=cfg["m"], k=cfg["k"], tau=cfg["tau"], seed=cfg["seed"],
                      sketch_prec="bf16x3", final_prec="bf16x3")
    theta, st = L.forward_state(A, p, handle=h)
    g = torch.empty_like(A)
    stream = torch.cuda.current_stream()

    def fwd():
        L.lev_sketch_dense(h, A, p, st["Atilde"])
        lib_rrqr_nosync(L, h, st["Atilde"], cfg["tau"], st["perm"], st["R"])
        L.lev_omega_factor(h, st["R"], st["perm"], st["d_rank"], cfg["d"], cfg["k"], cfg["seed"], L.LEV_OMEGA_REDUCED,
                           st["Mfull"])
        L.lev_final_dense(h, A, st["Mfull"], "bf16x3", theta)

    def bwd():
        L.lev_backward_dense(h, A, p, st["Atilde"], st["perm"], st["d_rank"], st["R"], st["Mfull"], w, g)

    res = {}
    for name, fn in (("forward_ms", fwd), ("backward_ms", bwd)):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        res[name] = a.elapsed_time(b) / reps
    res["bwd_over_fwd"] = res["backward_ms"] / res["forward_ms"]
    res["workload"] = "dense_2e5x64_backward (200,000 x 64, 5% rows x100; s=16384, m=256, k=128; split-BF16 forms)"
    return res


def lib_rrqr_nosync(L, h, At, tau, perm, R):
    import ctypes
    import torch
    m, d = At.shape
    L._check(L.lib.lev_rrqr(h.ptr, L._ptr(At), m, d, float(tau), L._ptr(perm), L._ptr(R), None,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))


if __name__ == "__main__":
    main()
