"""Device timeline of one mCQR2GS factorisation by phase, for the device call
(cqr_factor) and the host-buffer call (cqr_factor_host).

    python -m paper_2405_04237_gb300.phase_timeline --m 8388608 --n 1024 --b 128

Each phase the library reports through cqr_set_trace (Alg. 9 step 1 on the
first panel; per later panel the projection and update, CholeskyQR,
re-orthogonalisation, second CholeskyQR and R products) gets a CUDA event
recorded on the stream at its start and end, so the table shows when the
stream reached each phase and how long it ran.  For the host-buffer call the
difference to the device call is the copy time the overlap leaves exposed:
the first panel's copy in before the first phase, and the last panel's copy
out after the last one.  The input is a seeded Gaussian (the factorisation's
time does not depend on its condition number); host buffers are page-locked.
A pinned guard block is allocated before the host buffers (--no-guard
leaves it out).  A measurement utility: the factorisation runs in the CUDA
library.
"""
from __future__ import annotations

import argparse


def _timeline(fn, stream):
    import torch

    from . import _capi, load

    events = []

    def cb(name, panel, begin, ctx):
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        events.append((name.decode(), int(panel), int(begin), e))

    thunk = _capi.TRACE_FN(cb)
    L = load()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    L.cqr_set_trace(thunk, None)
    try:
        e0.record(stream)
        fn()
        e1.record(stream)
    finally:
        L.cqr_set_trace(_capi.TRACE_FN(), None)
    e1.synchronize()
    begins = [(n, p, e0.elapsed_time(e) / 1e3) for n, p, b, e in events if b]
    ends = [e0.elapsed_time(e) / 1e3 for n, p, b, e in events if not b]
    return [(n, p, t0, t1 - t0) for (n, p, t0), t1 in zip(begins, ends)], e0.elapsed_time(e1) / 1e3


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=1 << 23)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--b", type=int, default=128)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-guard", dest="guard", action="store_false",
                    help="allocate the host buffers without the pinned guard block before them")
    args = ap.parse_args(argv)

    import torch

    from . import empty_colmajor, empty_colmajor_pinned, factor, factor_host, load, workspace_size

    load()
    m, n, b = args.m, args.n, args.b
    g = torch.Generator(device="cuda")
    g.manual_seed(args.seed)
    A = torch.randn((n, m), generator=g, dtype=torch.float64, device="cuda").t()
    Q, R = empty_colmajor(m, n, "cuda"), empty_colmajor(n, n, "cuda")
    ws = torch.empty(workspace_size(m, n, b), dtype=torch.uint8, device="cuda")
    # a pinned guard block first: on GB300 the first ~8 GB of a process's
    # first large pinned allocation often copy at a tenth of the full rate,
    # which is a property of that host memory, not of the copies' schedule
    guard = torch.empty(16 << 27, dtype=torch.float64, pin_memory=True) if args.guard else None
    Ah, Qh, Rh = empty_colmajor_pinned(m, n), empty_colmajor_pinned(m, n), empty_colmajor_pinned(n, n)
    Ah.copy_(A)
    Qh.copy_(A)
    if guard is not None:
        gd = torch.empty(guard.numel(), dtype=torch.float64, device="cuda")
        gd.copy_(guard)
        guard.copy_(gd)
        del gd
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        factor(A, b, out=(Q, R), workspace=ws, stream=s)  # warm-up, status checked
        factor_host(Ah[:4 * n], b, stream=s)  # creates the library's copy stream
        dev, t_dev = _timeline(lambda: factor(A, b, out=(Q, R), workspace=ws, check=False, stream=s), s)
        host, t_host = _timeline(
            lambda: factor_host(Ah, b, out=(Qh, Rh), device_out=(Q, R), workspace=ws, check=False, stream=s), s)
    print(f"m={m} n={n} b={b}: device call {t_dev:.3f} s, host-buffer call {t_host:.3f} s "
          f"(+{1e3 * (t_host - t_dev):.1f} ms; {16 * m * n / 1e9:.1f} GB copied)")
    print(f"{'phase':18s} {'panel':>5s} | {'device start':>12s} {'dur':>7s} | {'host start':>10s} {'dur':>7s}")
    for (nm, p, sd, dd), (_, _, sh, dh) in zip(dev, host):
        print(f"{nm:18s} {p:5d} | {sd:12.3f} {dd:7.3f} | {sh:10.3f} {dh:7.3f}")
    print(f"after the last phase: device {t_dev - (dev[-1][2] + dev[-1][3]):.3f} s, "
          f"host {t_host - (host[-1][2] + host[-1][3]):.3f} s")


if __name__ == "__main__":
    main()
