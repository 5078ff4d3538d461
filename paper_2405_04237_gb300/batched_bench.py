"""Times the batched factorisation on a homogeneous batch (count matrices of
m x n, panel width b, the paper's test construction with kappa = 1e3).

    python -m paper_2405_04237_gb300.batched_bench --count 19 --m 20000 --n 128 --b 32 --group 8 [--pool]

Prints one line: schedule, seconds per batch (best of --reps, CUDA events)
and TFLOP/s (4 m n^2 per matrix).  A measurement utility; the factorisation
runs in the CUDA library.
"""
from __future__ import annotations

import argparse
import sys


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=19)
    ap.add_argument("--m", type=int, default=20000)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--b", type=int, default=32)
    ap.add_argument("--group", type=int, default=8)
    ap.add_argument("--pool", action="store_true", help="the stream-pool schedule instead of the persistent launch")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)

    import torch

    from . import batched_workspace_size, factor_batched, load

    try:
        from testmatrices import make_test_matrix_cuda
    except ImportError:  # run from the repository root
        sys.exit("run from the repository root (the test-matrix generator lives there)")
    load()
    base = make_test_matrix_cuda(args.m, args.n, 1e3, 77)
    As = [base.t().contiguous().t() for _ in range(args.count)]
    sched = "pool" if args.pool else "auto"
    ms, ns, bs = [args.m] * args.count, [args.n] * args.count, [args.b] * args.count
    ws = torch.empty(batched_workspace_size(ms, ns, bs, schedule=sched, group=args.group), dtype=torch.uint8,
                     device="cuda")
    st = torch.zeros(args.count, dtype=torch.int32, device="cuda")
    factor_batched(As, bs, workspace=ws, status=st, schedule=sched, group=args.group)  # warm-up, statuses checked
    best = float("inf")
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        factor_batched(As, bs, check=False, workspace=ws, status=st, schedule=sched, group=args.group)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    flops = args.count * 4.0 * args.m * args.n * args.n
    print(f"{sched} count={args.count} m={args.m} n={args.n} b={args.b} G={args.group}: "
          f"{best * 1e3:.2f} ms  {flops / best / 1e12:.4f} TFLOP/s", flush=True)


if __name__ == "__main__":
    main()
