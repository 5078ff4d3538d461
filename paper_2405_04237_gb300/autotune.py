"""Panel-width autotuner.

The panel width b is the method's one tuning knob (Sec. 5.3, Sec. 6): smaller
panels lower each panel's condition number (Eq. cond_bounds) and so decide
stability; otherwise b only moves time between kernels, since mCQR2GS costs
4 m n^2 flops for every b.  The tuner therefore
  1. keeps only widths b | n whose panel count k = n/b meets the stability
     floor for the caller's condition-number estimate (mCQR2GS: 1 panel up to
     1e7, 2 up to 1e11, 3 beyond -- Sec. 5.4, Fig. 6; CQR2GS: 1 panel up to
     1e7, 4 up to 1e11, 10 beyond -- Sec. 5.3, Fig. 3), and
  2. times the remaining candidates on a probe matrix of the same n and
     min(m, 2^20) rows, and returns the fastest.
Results are cached per (GPU name, n, variant, m bucket) in a JSON file next
to the built library.

autotune_batched() tunes the persistent batched launch the same way, on the
caller's own batch: the CTAs per matrix G (the launch's tile shape: how many
SMs split one matrix's rows) and the starting panel count (every matrix
starts with b_i = n_i / k0), each candidate timed with the adaptive panel
width switched on -- a panel that is too ill-conditioned is narrowed on the
device (Sec. 5.3-5.4) -- so no condition-number estimate is needed.  The
fastest candidate whose every status is 0 wins.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import build as _build

_CACHE = os.path.join(_build.BUILD, "autotune.json")


def min_panels(variant: str, kappa: float | None) -> int:
    if kappa is None:
        kappa = 1e16
    if variant == "mcqr2gs":
        return 1 if kappa <= 1e7 else (2 if kappa <= 1e11 else 3)
    if variant == "cqr2gs":
        return 1 if kappa <= 1e7 else (4 if kappa <= 1e11 else 10)
    return 1


def candidates(n: int, variant: str = "mcqr2gs", kappa: float | None = None, lo: int = 16, hi: int = 256):
    kmin = min_panels(variant, kappa)
    c = [b for b in range(1, n + 1) if n % b == 0 and n // b >= kmin and b <= hi and (b >= lo or b == n)]
    if not c:
        c = [max(b for b in range(1, n + 1) if n % b == 0 and n // b >= kmin)]
    return c


def _load_cache() -> dict:
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(c: dict) -> None:
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    tmp = _CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE)


def autotune(m: int, n: int, variant: str = "mcqr2gs", kappa: float | None = None, cands=None, reps: int = 2,
             use_cache: bool = True, verbose: bool = False) -> int:
    """The fastest stable panel width for an m x n factorisation."""
    from . import empty_colmajor, factor, workspace_size

    cands = list(cands) if cands is not None else candidates(n, variant, kappa)
    if len(cands) == 1:
        return cands[0]
    dev = torch.cuda.get_device_name()
    mb = int(math.log2(max(m, 2)))
    key = f"{dev}|n={n}|{variant}|m2^{mb}|k>={min_panels(variant, kappa)}|{','.join(map(str, cands))}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return int(cache[key]["b"])
    mp = int(min(m, 1 << 20))
    g = torch.Generator(device="cuda")
    g.manual_seed(12345)
    A = torch.randn((n, mp), generator=g, dtype=torch.float64, device="cuda").t()  # column-major, kappa ~ 1
    Q = empty_colmajor(mp, n, "cuda")
    R = empty_colmajor(n, n, "cuda")
    times = {}
    for b in cands:
        ws = torch.empty(workspace_size(mp, n, b, variant), dtype=torch.uint8, device="cuda")
        factor(A, b, variant, out=(Q, R), workspace=ws)  # warm-up + status check
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            factor(A, b, variant, out=(Q, R), workspace=ws, check=False)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        times[b] = best
        if verbose:
            print(f"autotune n={n} {variant} b={b}: {best:.3f} ms", flush=True)
        del ws
    bbest = min(times, key=times.get)
    if use_cache:
        cache = _load_cache()
        cache[key] = {"b": bbest, "ms": times, "m_probe": mp}
        _save_cache(cache)
    return bbest


def _batch_key(As, variant):
    ns = sorted({int(A.shape[1]) for A in As})
    hist = ",".join(f"{n}:{sum(1 for A in As if A.shape[1] == n)}:{int(math.log2(max(2, sum(A.shape[0] for A in As if A.shape[1] == n))))}"
                    for n in ns)
    return f"{torch.cuda.get_device_name()}|batched|{variant}|{len(As)}|{hist}"


def starting_panels(ns, k0):
    """b_i = n_i / k0 where that is a multiple of 4 dividing n_i, else the
    nearest such width below it (at least 4, at most n_i)."""
    out = []
    for n in ns:
        b = max(4, n // k0)
        while b > 4 and (n % b or b % 4):
            b -= 1
        out.append(min(b, n))
    return out


def autotune_batched(As, variant: str = "mcqr2gs", groups=(4, 8, 19), panel_counts=(1, 2, 4), reps: int = 2,
                     use_cache: bool = True, verbose: bool = False):
    """(G, panel_b list) for the persistent batched launch of these matrices."""
    from . import batched_workspace_size, factor_batched

    ns = [int(A.shape[1]) for A in As]
    ms = [int(A.shape[0]) for A in As]
    key = _batch_key(As, variant)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return int(cache[key]["G"]), starting_panels(ns, int(cache[key]["k0"]))
    best, times = None, {}
    for k0 in panel_counts:
        bs = starting_panels(ns, k0)
        for G in groups:
            ws = torch.empty(batched_workspace_size(ms, ns, bs, variant, group=G, halving=True), dtype=torch.uint8,
                             device="cuda")
            st = torch.zeros(len(As), dtype=torch.int32, device="cuda")
            factor_batched(As, bs, variant, workspace=ws, status=st, group=G, halving=True, check=False)
            torch.cuda.synchronize()
            if int((st != 0).sum()) != 0:
                continue
            t = float("inf")
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                factor_batched(As, bs, variant, workspace=ws, status=st, group=G, halving=True, check=False)
                e1.record()
                e1.synchronize()
                t = min(t, e0.elapsed_time(e1))
            times[f"k0={k0},G={G}"] = t
            if verbose:
                print(f"autotune batched k0={k0} G={G}: {t:.2f} ms", flush=True)
            if best is None or t < best[0]:
                best = (t, G, k0)
            del ws
    if best is None:
        raise RuntimeError("autotune_batched: no candidate factored every matrix")
    if use_cache:
        cache = _load_cache()
        cache[key] = {"G": best[1], "k0": best[2], "ms": times}
        _save_cache(cache)
    return best[1], starting_panels(ns, best[2])
