"""ctypes binding of the C ABI declared in ``include/cqr.h``.

Argument marshalling only: every step of a factorisation runs in the CUDA
library ``_build/libcqr_gb300.so``.  There is no CPU fallback: if the library
is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

MCQR2GS, CQR2GS, CQR2, SCQR3 = 0, 1, 2, 3
LOOKAHEAD = 0x100
ADAPTIVE = 0x200
EMULATED = 0x400
HALVE = 0x800
BATCH_POOL = 0x1000


def BATCH_GROUP(G: int) -> int:
    return int(G) << 16
VARIANTS = {"mcqr2gs": MCQR2GS, "cqr2gs": CQR2GS, "cqr2": CQR2, "scqr3": SCQR3}
ERR_CUDA = -1000
STATUS_TIMEOUT = -2000
ERR_NOALLOC_TOO_LARGE = -3000
ERR_ALLOC = -4000
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
TRACE_FN = ctypes.CFUNCTYPE(None, ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p)
NOALLOC_SCRATCH_BYTES = 64 << 20

EXPORTS = [
    "cqr_workspace_size", "cqr_default_panel", "cqr_factor", "cqr_read_status", "cqr_read_panel_width", "cqr_set_allocator",
    "cqr_backward_workspace_size", "cqr_backward", "cqr_batched_workspace_size",
    "cqr_factor_batched", "cqr_status_string", "cqr_probe_fp64_peak", "cqr_probe_fp64",
    "cqr_factor_noalloc", "cqr_factor_host", "cqr_test_arm_wait_expiry", "cqr_test_arm_barrier_expiry", "cqr_batched_panel_widths", "cqr_launch_count", "cqr_set_trace", "cqr_profile_enable", "cqr_profile_disable", "cqr_profile_read", "cqr_kernel_class_name",
]
KERNEL_CLASSES = ["gram_syrk", "projection_tn", "split_reduce", "cholesky", "trsm", "update_gemm", "misc",
                  "batched"]


class CQRError(RuntimeError):
    """Argument error or numerical breakdown reported by the CUDA library."""

    def __init__(self, code: int, what: str):
        self.code = int(code)
        super().__init__(f"{what}: {self.code} ({status_string(self.code)})")


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        L = ctypes.CDLL(path)
        i64, vp, sz, c_int, dp = ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p
        P64 = ctypes.POINTER(ctypes.c_int64)
        PI = ctypes.POINTER(ctypes.c_int)
        PV = ctypes.POINTER(ctypes.c_void_p)
        sigs = {
            "cqr_workspace_size": (sz, [i64, i64, c_int, c_int]),
            "cqr_default_panel": (c_int, [i64]),
            "cqr_factor": (c_int, [i64, i64, dp, i64, c_int, dp, i64, dp, i64, c_int, vp, sz, vp]),
            "cqr_read_status": (c_int, [vp, vp, PI]),
            "cqr_read_panel_width": (c_int, [vp, vp, PI]),
            "cqr_set_allocator": (c_int, [ALLOC_FN, FREE_FN, vp]),
            "cqr_factor_noalloc": (c_int, [i64, i64, dp, i64, c_int, dp, i64, dp, i64, c_int, vp, vp]),
            "cqr_factor_host": (c_int, [i64, i64, dp, i64, c_int, dp, i64, dp, i64, c_int, dp, i64, dp, i64, vp, sz, vp]),
            "cqr_backward_workspace_size": (sz, [i64, i64]),
            "cqr_backward": (c_int, [i64, i64, dp, i64, dp, i64, dp, i64, dp, i64, dp, i64, vp, sz, vp]),
            "cqr_batched_workspace_size": (sz, [c_int, P64, P64, PI, c_int]),
            "cqr_factor_batched": (c_int, [c_int, P64, P64, P64, PI, PV, PV, PV, c_int, vp, vp, sz, vp]),
            "cqr_status_string": (ctypes.c_char_p, [c_int]),
            "cqr_probe_fp64_peak": (ctypes.c_double, [c_int]),
            "cqr_probe_fp64": (c_int, [c_int, c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
            "cqr_test_arm_wait_expiry": (c_int, [c_int, c_int, ctypes.c_longlong]),
            "cqr_test_arm_barrier_expiry": (c_int, [c_int, c_int, c_int, ctypes.c_longlong]),
            "cqr_batched_panel_widths": (c_int, [c_int, vp, vp, PI]),
            "cqr_launch_count": (ctypes.c_ulonglong, []),
            "cqr_set_trace": (c_int, [TRACE_FN, vp]),
            "cqr_profile_enable": (c_int, [c_int]),
            "cqr_profile_disable": (c_int, []),
            "cqr_profile_read": (c_int, [c_int, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]),
            "cqr_kernel_class_name": (ctypes.c_char_p, [c_int]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def status_string(code: int) -> str:
    return load().cqr_status_string(int(code)).decode()
