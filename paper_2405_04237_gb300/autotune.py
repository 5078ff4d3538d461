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
