#!/usr/bin/env python
"""Benchmark: mCQR2GS FP64 TFLOP/s on one GB300 (plus batched and adjoint).

One step = one mCQR2GS factorisation (Alg. 9) of the m = 2^23, n = 1024,
kappa = 1e15 test matrix A = U diag(sigma) V^T (Sec. 2.2 construction,
seeded, synthetic), out of place (A is read, Q and R are written), panel
width b = 128 (the autotuner, --panel 0, finds 64, 128 and 256 within 0.3 %
of one another on this shape and picks among them by noise; the fixed width
keeps runs comparable).  Rate = 4 m n^2 / t,
the paper's flop convention for mCQR2GS (Table 2 with the final R product
removed, Sec. 5.4).  The matrix (68.7 GB) is far larger than L2, so no L2
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle on the host cores (a bounded row
sample of the same workload) and prints the same JSON line with
"impl": "reference".  With --gpus N > 1 (under torchrun) every rank factors
its own replica (replicas only: the library has no multi-GPU path) and the
value is the sum over ranks of the work divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mCQR2GS FP64 TFLOP/s; batched QR/s vs looped; at ‖I−QᵀQ‖_F≤1e-13"
M_FULL, N_FULL, KAPPA_FULL, SEED_FULL = 1 << 23, 1024, 1e15, 1002
PANEL_CANDIDATES = (64, 128, 256)
N_SM = 152
# probe iterations: about 0.2-0.3 s per probe launch on GB300
PROBE_ITERS = {"dfma": 100000, "dmma_m8n8k4": 30000, "dmma_m16n8k16": 4000}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    # --rows / --cols: the same, for launchers (torch.distributed.run) that read --m / --n as their own prefixes
    p.add_argument("--m", "--rows", dest="m", type=int, default=M_FULL)
    p.add_argument("--n", "--cols", dest="n", type=int, default=N_FULL)
    p.add_argument("--kappa", type=float, default=KAPPA_FULL)
    p.add_argument("--panel", type=int, default=128, help="panel width; 0 = autotune among 64/128/256")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the batched and adjoint sub-benchmarks")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--no-check", action="store_true", help="skip the accuracy norms")
    p.add_argument("--emulated", action="store_true",
                   help="time the emulated variant (projections on FP8 tensor cores) instead of native FP64")
    return p.parse_args()


# --------------------------------------------------------------------------- distributed plumbing
def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        return dist, dist.get_rank(), ws
    return None, 0, 1


def _reduce_device(dist):
    # NCCL reduces device tensors; gloo (the reference arm, CPU tests) host tensors
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def allreduce_max(dist, x):
    """Maximum of x over the ranks (timing only: not on the data path)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(dist, x):
    """Sum of x over the ranks (launch counts only)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=10)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- CPU baseline (oracle)
def oracle_sample(n, b, kappa, target_s, cap_rows=1 << 18):
    """A row sample of the workload (same n, b, kappa construction) sized so
    that one oracle mCQR2GS on it takes about target_s seconds (between
    target_s / 2 and target_s when the row cap allows).

    The oracle runs its row sums in parallel over fixed 4096-row blocks, so
    its time grows linearly with the rows only once every thread has a
    block: the probe uses 4096 rows per thread, is run once untimed (thread
    start-up, page faults), and is scaled up by doublings from there."""
    import oracle
    from testmatrices import make_test_matrix

    oracle.build()
    m_s = min(cap_rows, (1 << 12) * max(1, oracle.num_threads()))
    A = make_test_matrix(m_s, n, kappa, seed=SEED_FULL)
    oracle.mcqr2gs(A, b, check=False)
    t0 = time.perf_counter()
    oracle.mcqr2gs(A, b, check=False)
    dt = time.perf_counter() - t0
    while dt * 2 <= target_s and m_s * 2 <= cap_rows:
        m_s *= 2
        dt *= 2
    if A.shape[0] != m_s:
        A = make_test_matrix(m_s, n, kappa, seed=SEED_FULL)
    return A


def time_oracle(A, b):
    import oracle

    t0 = time.perf_counter()
    oracle.mcqr2gs(A, b, check=False)
    dt = time.perf_counter() - t0
    m_s, n = A.shape
    return 4.0 * m_s * n * n / dt / 1e12, dt


def cpu_baseline(n, b, kappa, target_s=20.0):
    """The oracle timed on the host cores on a bounded row sample."""
    import oracle

    A = oracle_sample(n, b, kappa, target_s)
    v, dt = time_oracle(A, b)
    desc = (f"oracle mCQR2GS (Alg. 9, plain C, OpenMP) on a {A.shape[0]} x {n} row sample of the same "
            f"construction (kappa={kappa:.0e}, b={b}), one run of {dt:.1f} s")
    return v, desc, oracle.num_threads(), dt, A.shape[0]


def workload_config(m, n, kappa, b, emu, world):
    """The "config" object of the JSON line (the same for both arms)."""
    return {"workload": f"mCQR2GS m={m} n={n} kappa={kappa:.0e} b={b} (out of place)"
                        + (", products emulated on FP8 tensor cores" if emu else ""), "m": m, "n": n,
            "kappa": kappa, "panel_b": b, "variant": "mcqr2gs",
            "l2": f"inputs larger than L2 ({8 * m * n / 1e9:.1f} GB), no flush",
            "parallelism": "replicas" if world > 1 else "single-gpu"}


def run_reference(args, dist, rank, world):
    if rank != 0:
        return
    import oracle

    b = args.panel or 128
    A = oracle_sample(args.n, b, args.kappa, target_s=8.0)
    steps = []
    for i in range(args.warmup + args.steps):
        v, dt = time_oracle(A, b)
        if i >= args.warmup:
            steps.append((v, dt))
    v = statistics.median(x[0] for x in steps)
    m_s = A.shape[0]
    desc = (f"oracle mCQR2GS (Alg. 9, plain C, OpenMP) on a {m_s} x {args.n} row sample of the workload "
            f"(kappa={args.kappa:.0e}, b={b}); rate scaled by the flop count 4 m n^2 of the sample")
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": v,
        "unit": "TFLOP/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(x[1] for x in steps),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {**workload_config(args.m, args.n, args.kappa, b, False, world), "sample_rows": m_s},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------- our arm
def accuracy(A, Q, R, chunk=1 << 20):
    """||I - Q^T Q||_F, ||A - Q R||_F / ||A||_F with torch FP64 GEMMs (row chunks)."""
    import torch

    m, n = Q.shape
    G = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    rs2 = torch.zeros((), dtype=torch.float64, device="cuda")
    a2 = torch.zeros((), dtype=torch.float64, device="cuda")
    for r0 in range(0, m, chunk):
        r1 = min(m, r0 + chunk)
        Qc = Q[r0:r1]
        G += Qc.t() @ Qc
        D = A[r0:r1] - Qc @ R
        rs2 += (D * D).sum()
        a2 += (A[r0:r1] * A[r0:r1]).sum()
    orth = torch.linalg.norm(torch.eye(n, dtype=torch.float64, device="cuda") - G).item()
    return orth, (rs2.sqrt() / a2.sqrt()).item()


def bench_batched(P, peak_tflops):
    """Batched workload: 512 matrices, m in [2000, 200000], n in {16..128},
    kappa log-uniform in [1e2, 1e15], as ONE persistent launch replayed from
    a CUDA graph.  The autotuner picks the CTAs per matrix and the starting
    panel count on this batch, with the adaptive panel width on (rejected
    panels are narrowed on the device), so no condition number is used.
    Compared with a loop of single calls and with the stream-pool schedule,
    both at the final panel widths the launch arrived at; matrices/s, and
    per width class n the persistent launch on that class alone."""
    import torch

    from paper_2405_04237_gb300.autotune import autotune_batched
    from testmatrices import batch_specs, make_test_matrix_cuda

    specs = batch_specs(512)
    As = [make_test_matrix_cuda(m, n, k, s, chunk_rows=1 << 18) for (m, n, k, s) in specs]
    torch.cuda.synchronize()
    flops = sum(4.0 * A.shape[0] * A.shape[1] ** 2 for A in As)

    def timed(fn, reps=3):
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return best

    G, bs = autotune_batched(As)
    g = P.BatchedGraph(As, bs, group=G, halving=True)
    g.replay()
    torch.cuda.synchronize()
    tg = timed(g.replay)
    bad = int((g.status != 0).sum().item())
    widths = P.batched_panel_widths(g.workspace, len(As))
    # accuracy of every member (torch FP64 GEMMs)
    orth = resid = 0.0
    for (Q, R), A in zip(g.out, As):
        n = Q.shape[1]
        orth = max(orth, torch.linalg.norm(torch.eye(n, dtype=torch.float64, device="cuda") - Q.t() @ Q).item())
        resid = max(resid, (torch.linalg.norm(A - Q @ R) / torch.linalg.norm(A)).item())
    # looped single calls at the same final widths (workspaces allocated up front)
    Qs = [P.empty_colmajor(A.shape[0], A.shape[1], "cuda") for A in As]
    Rs = [P.empty_colmajor(A.shape[1], A.shape[1], "cuda") for A in As]
    wss = [torch.empty(P.workspace_size(A.shape[0], A.shape[1], b), dtype=torch.uint8, device="cuda")
           for A, b in zip(As, widths)]

    def loop():
        for A, b, Q, R, w in zip(As, widths, Qs, Rs, wss):
            P.factor(A, b, out=(Q, R), workspace=w, check=False)

    loop()
    torch.cuda.synchronize()
    tl = timed(loop)
    del wss, Qs, Rs
    gp = P.BatchedGraph(As, widths, schedule="pool")
    gp.replay()
    torch.cuda.synchronize()
    tp = timed(gp.replay)
    del gp
    # per width class: the persistent launch on that class alone
    per_n = {}
    for n in sorted({A.shape[1] for A in As}):
        idx = [i for i, A in enumerate(As) if A.shape[1] == n]
        sub = [As[i] for i in idx]
        sb = [bs[i] for i in idx]
        fl = sum(4.0 * A.shape[0] * A.shape[1] ** 2 for A in sub)
        gs = P.BatchedGraph(sub, sb, group=G, halving=True)
        gs.replay()
        torch.cuda.synchronize()
        ts = timed(gs.replay)
        per_n[str(n)] = {"matrices": len(sub), "share_of_flops": fl / flops, "seconds": ts,
                         "tflops": fl / ts / 1e12, "frac_of_fp64_peak": fl / ts / 1e12 / peak_tflops}
        del gs
    return {"matrices": len(As), "schedule": "one persistent cooperative launch (CUDA-graph replay)",
            "batched_graph_qr_per_s": len(As) / tg, "batched_graph_tflops": flops / tg / 1e12,
            "batched_frac_of_fp64_peak": flops / tg / 1e12 / peak_tflops,
            "looped_qr_per_s": len(As) / tl, "looped_tflops": flops / tl / 1e12,
            "speedup_vs_looped": tl / tg, "pool_graph_qr_per_s": len(As) / tp,
            "autotune": {"ctas_per_matrix": G, "starting_panels_hist": {str(b): bs.count(b) for b in sorted(set(bs))}},
            "final_panels_hist": {str(b): widths.count(b) for b in sorted(set(widths))},
            "max_orth_fro": orth, "max_resid_rel": resid, "failed_status": bad, "per_n": per_n,
            "workload": "512 matrices, m U[2000,200000], n in {16,32,64,128}, kappa log-U[1e2,1e15]; "
                        "panel widths from the autotuner + on-device adaptive width (no kappa used)"}


def bench_adjoint(P):
    """Forward + hand-written adjoint at m = 2^20, n = 128, kappa = 1e8."""
    import torch

    from testmatrices import make_test_matrix_cuda

    m, n = 1 << 20, 128
    A = make_test_matrix_cuda(m, n, 1e8, 1004)
    g = torch.Generator(device="cuda")
    g.manual_seed(1005)
    dQ = torch.randn((n, m), generator=g, dtype=torch.float64, device="cuda").t()
    dR = torch.triu(torch.randn((n, n), generator=g, dtype=torch.float64, device="cuda"))
    b = 64
    Q, R = P.factor(A, b)
    P.backward(Q, R, dQ, dR)
    torch.cuda.synchronize()
    tf, tb = [], []
    for _ in range(3):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        Q, R = P.factor(A, b, check=False)
        e1.record()
        P.backward(Q, R, dQ, dR)
        e2.record()
        e2.synchronize()
        tf.append(e0.elapsed_time(e1))
        tb.append(e1.elapsed_time(e2))
    f, bw = min(tf), min(tb)
    return {"m": m, "n": n, "panel_b": b, "forward_ms": f, "backward_ms": bw, "backward_over_forward": bw / f,
            "forward_tflops": 4.0 * m * n * n / f / 1e9, "backward_tflops": 5.0 * m * n * n / bw / 1e9}


def bench_emulated(P, A, Q, R, b, args, flops, t_native):
    """The same workload with the m-row projections on the FP8 tensor cores
    (FP64-accurate Ozaki splitting, CQR_EMULATED): one warm-up with status
    check, then timed steps, then the accuracy norms."""
    import torch

    m, n = A.shape
    ws = torch.empty(P.workspace_size(m, n, b, "mcqr2gs", emulated=True), dtype=torch.uint8, device="cuda")
    P.factor(A, b, out=(Q, R), workspace=ws, emulated=True)
    steps = max(1, min(args.steps, 2))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        P.factor(A, b, out=(Q, R), workspace=ws, emulated=True, check=False)
    e1.record()
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / steps
    status = P.read_status(ws)
    orth, res = accuracy(A, Q, R)
    return {"value": flops / t / 1e12, "unit": "TFLOP/s (FP64-equivalent, 4 m n^2 / t)", "ms_per_step": 1e3 * t,
            "speedup_vs_native": t_native / t, "orth_fro": orth, "resid_rel": res, "status": status,
            "what": "Gram matrices, projections, updates and the triangular solves' coupling products on the "
                    "tcgen05 FP8 tensor cores (14-digit Ozaki splitting, exact FP32 level sums in TMEM); "
                    "Cholesky factorisations and the solves' 32-column substitutions native FP64"}


# DRAM bytes per launch of the update kernel class, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of every update launch of an
# m = 2^18, n = 1024, b = 128 factorisation: 33.29 GB over 45 launches,
# scaled by m (every launch that matters streams m-row operands).
UPDATE_DRAM_BYTES_PER_LAUNCH_2P18 = 33.29e9 / 45


def update_traffic(m, n, b, dom, emulated):
    if dom != "update_gemm" or emulated or n != 1024 or b != 128:
        return None
    return UPDATE_DRAM_BYTES_PER_LAUNCH_2P18 * m / 2 ** 18


def run_ours(args, dist, rank, world):
    import torch

    import paper_2405_04237_gb300 as P
    from paper_2405_04237_gb300.autotune import autotune
    from testmatrices import make_test_matrix_cuda

    P.load()
    dev = torch.cuda.current_device()
    m, n, kappa = args.m, args.n, args.kappa
    b = args.panel or autotune(m, n, "mcqr2gs", kappa, cands=[c for c in PANEL_CANDIDATES if n % c == 0 and n // c >= 3])
    # Q, R and the workspace first: the generator's dense QR of a 2^23 x 1024
    # Gaussian leaves device memory in a state where a buffer allocated after
    # it has regions the copy engines reach at a tenth of their rate (measured
    # on GB300), and Q is the device buffer of the host-buffer leg below.
    Q = P.empty_colmajor(m, n, "cuda")
    R = P.empty_colmajor(n, n, "cuda")
    emu = bool(args.emulated)
    ws = torch.empty(P.workspace_size(m, n, b, "mcqr2gs", emulated=emu), dtype=torch.uint8, device="cuda")
    A = make_test_matrix_cuda(m, n, kappa, SEED_FULL + 100 * rank)
    torch.cuda.synchronize()
    for i in range(args.warmup):
        P.factor(A, b, out=(Q, R), workspace=ws, check=(i == 0), emulated=emu)
    torch.cuda.synchronize()
    # FP64 peak microbenchmarks (clocks are warm now): DFMA and the two
    # mma.sync .f64 shapes, each as flop per SM clock cycle
    probes = {k: P.probe_fp64(k, it) for k, it in PROBE_ITERS.items()}
    best_probe = max(probes.values(), key=lambda r: r["flop_per_clk_sm"])
    stream = torch.cuda.current_stream()
    barrier(dist)
    torch.cuda.synchronize()
    l0 = P.launch_count()
    with ClockSampler(dev) as clk, P.KernelTimer(100000) as kt:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            P.factor(A, b, out=(Q, R), workspace=ws, check=False, stream=stream, emulated=emu)
        e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize()
    barrier(dist)
    launches = P.launch_count() - l0
    t_step = e0.elapsed_time(e1) / 1e3 / args.steps
    status = P.read_status(ws)
    t_max = allreduce_max(dist, t_step)
    launches_all = int(allreduce_sum(dist, launches))
    flops = 4.0 * m * n * n
    value = world * flops / t_max / 1e12
    prof = kt.read()
    clocks = clk.summary()

    # dominant kernel (largest device time) and its roofline
    dom = max(prof, key=lambda k: prof[k]["ms"])
    tot_ms = sum(v["ms"] for v in prof.values())
    # measured peak: the best probe's flop/clk/SM x SMs x the SM clock sampled in the timed region
    clk_mhz = clocks["sm_mhz"] or best_probe["sm_mhz"]
    peak = best_probe["flop_per_clk_sm"] * N_SM * clk_mhz * 1e6 / 1e12
    ach = prof[dom]["flops"] / (prof[dom]["ms"] * 1e-3) / 1e12 if prof[dom]["ms"] > 0 else 0.0
    roofline = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": update_traffic(m, n, b, dom, emu), "kernel": dom,
                "peak_note": (f"measured: FP64 {best_probe['kind']} microbenchmark "
                              f"{best_probe['flop_per_clk_sm']:.3f} flop/clk/SM x {N_SM} SMs x {clk_mhz:.0f} MHz "
                              "(median SM clock sampled during the timed region); probes: "
                              + ", ".join(f"{k} {v['flop_per_clk_sm']:.3f} flop/clk/SM = {v['gflops'] / 1e3:.4f} "
                                          f"TFLOP/s at {v['sm_mhz']:.0f} MHz" for k, v in probes.items())),
                "share_of_device_time": prof[dom]["ms"] / tot_ms if tot_ms else None,
                "launches": prof[dom]["launches"]}
    kernels = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps,
                   "share": v["ms"] / tot_ms if tot_ms else None,
                   "tflops": (v["flops"] / (v["ms"] * 1e-3) / 1e12) if v["ms"] > 0 else None}
               for k, v in prof.items() if v["launches"]}

    acc = {}
    if not args.no_check:
        orth, res = accuracy(A, Q, R)
        acc = {"orth_fro": orth, "orth_fro_over_sqrt_n": orth / n ** 0.5, "resid_rel": res, "status": status}

    # end to end through the host-buffer entry point (cqr_factor_host): A in
    # pinned host memory, Q and R back to pinned host memory, every copy
    # inside the timed region (overlapped with the panels by the library)
    e2e = None
    if not args.no_e2e:
        # A pinned guard block first.  Measured on GB300: in most runs the
        # first ~8 GB of a process's first large pinned allocation copy at
        # 20-80 GB/s instead of 210, and the first panel of A, whose copy the
        # factorisation waits for, would sit there; behind a guard it copies
        # at full rate.  The guard is touched once by a copy each way, as in
        # the measurement.
        guard_n = 16 << 27  # 16 GiB of FP64: the slow region is ~8 GB whatever the matrix size
        why = ""
        try:
            guard = torch.empty(guard_n, dtype=torch.float64, pin_memory=True)
            Ah = P.empty_colmajor_pinned(m, n)
            Qh = P.empty_colmajor_pinned(m, n)
            Rh = P.empty_colmajor_pinned(n, n)
        except (RuntimeError, MemoryError) as ex:  # not enough page-locked host memory
            guard = Ah = Qh = Rh = None
            why = str(ex).splitlines()[0][:160] if str(ex) else type(ex).__name__
        # every rank takes the same decision before the barrier below
        if allreduce_max(dist, 1.0 if why else 0.0) > 0.0:
            e2e = {"value": None, "unit": "TFLOP/s", "h2d_bytes_per_step": 8 * m * n,
                   "d2h_bytes_per_step": 8 * (m * n + n * n),
                   "unavailable": "page-locked host buffers could not be allocated on every rank"
                                  + (f" ({why})" if why else "")}
            del guard, Ah, Qh, Rh
    if not args.no_e2e and e2e is None:
        Ah.copy_(A)
        Qh.copy_(A)
        gd = torch.empty(guard_n, dtype=torch.float64, device="cuda")
        gd.copy_(guard)
        guard.copy_(gd)
        del gd
        P.factor_host(Ah[:4 * n], b, stream=stream, emulated=emu)  # creates the library's copy stream
        barrier(dist)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            P.factor_host(Ah, b, out=(Qh, Rh), device_out=(Q, R), workspace=ws, check=False, stream=stream,
                          emulated=emu)
        e1.record(stream)
        e1.synchronize()
        t_e2e = allreduce_max(dist, e0.elapsed_time(e1) / 1e3 / args.steps)
        e2e = {"value": world * flops / t_e2e / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": 8 * m * n,
               "d2h_bytes_per_step": 8 * (m * n + n * n), "ms_per_step": 1e3 * t_e2e,
               "api": "cqr_factor_host (pinned host A, Q, R; copies overlapped with the panel loop)",
               "status": P.read_status(ws, stream)}
        if not args.no_check:  # the host result is the device result
            e2e["host_equals_device"] = bool(torch.equal(Qh[:4096], Q[:4096].cpu()) and torch.equal(Rh, R.cpu()))
        del Ah, Qh, Rh, guard

    extras = {}
    if not args.no_extras and not emu and rank == 0:
        extras["emulated"] = bench_emulated(P, A, Q, R, b, args, flops, t_step)
    del A, Q, R, ws
    torch.cuda.empty_cache()
    if not args.no_extras and rank == 0:
        extras["batched"] = bench_batched(P, peak)
        torch.cuda.empty_cache()
        extras["adjoint"] = bench_adjoint(P)
        torch.cuda.empty_cache()

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        v, desc, threads, dt, m_s = cpu_baseline(n, b, kappa)
        cpu = {"value": v, "unit": "TFLOP/s", "cores": threads, "kind": "oracle", "sample": desc, "seconds": dt}

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value,
            "unit": "TFLOP/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1e3 * t_max,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(m, n, kappa, b, emu, world),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_all,
            "clocks": clocks,
            "accuracy": acc,
            "kernels": kernels,
            "fp64_probes": probes,
            **extras,
        }
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    dist, rank, world = dist_init(args)
    try:
        if args.impl == "reference":
            run_reference(args, dist, rank, world)
        else:
            run_ours(args, dist, rank, world)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
