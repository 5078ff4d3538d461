"""CPU FP64 oracle for CholeskyQR2-with-Gram-Schmidt QR factorisations.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow statement of the
arithmetic of arXiv 2405.04237 (Alg. 1, 3, 4, 5, 6, 7, 9) plus the adjoint of
A = QR.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code with the CUDA library
(``paper_2405_04237_gb300``) and never imports it; the CUDA library never
imports this package.

Every routine takes and returns numpy FP64 arrays.  Internally the C code
works on column-major (Fortran-order) copies, so callers can pass any layout.

Parity pins (what fixes each routine independently of itself) live in
``tests/test_oracle_pins.py``: the exact QR of dyadic inputs (closed form),
Householder QR by brute force on tiny inputs, closed forms (R_11 = ||a_1||,
orthogonal columns give a diagonal R, the shifted CholeskyQR of exactly
orthonormal columns gives sqrt(1 + s) I), the b = n reductions, the paper's
stability claims (Sec. 4, Sec. 5.3-5.4) on scaled-down matrices, and finite
differences / torch autograd for the adjoint.  ``tests/test_oracle_mutations.py``
checks that those pins reject mutated copies of the C source.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cqr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcqr_oracle.so")
_lock = threading.Lock()
_lib = None

LITERAL_R = 1  # or_mcqr2gs flag: drop the R_{1:j-1,j} += Z S1 term
ADAPTIVE = 2   # or_mcqr2gs flag: runtime choice of the second CholeskyQR pass (Sec. 7)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _sigs():
    i64, dp, cdp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)
    return {
        "or_set_block_rows": (None, [i64]),
        "or_get_block_rows": (i64, []),
        "or_num_threads": (ctypes.c_int, []),
        "or_gram": (None, [i64, i64, cdp, i64, dp, i64]),
        "or_tn": (None, [i64, i64, i64, cdp, i64, cdp, i64, dp, i64]),
        "or_chol": (ctypes.c_int, [i64, cdp, i64, dp, i64]),
        "or_trsm": (None, [i64, i64, dp, i64, cdp, i64]),
        "or_update": (None, [i64, i64, i64, dp, i64, cdp, i64, cdp, i64]),
        "or_cqr": (ctypes.c_int, [i64, i64, dp, i64, dp, i64]),
        "or_scqr": (ctypes.c_int, [i64, i64, dp, i64, dp, i64]),
        "or_cqr2": (ctypes.c_int, [i64, i64, dp, i64, dp, i64]),
        "or_scqr3": (ctypes.c_int, [i64, i64, dp, i64, dp, i64]),
        "or_cqrgs": (ctypes.c_int, [i64, i64, i64, dp, i64, dp, i64]),
        "or_cqr2gs": (ctypes.c_int, [i64, i64, i64, dp, i64, dp, i64]),
        "or_mcqr2gs": (ctypes.c_int, [i64, i64, i64, dp, i64, dp, i64, ctypes.c_int]),
        "or_mcqr2gs_halving": (ctypes.c_int, [i64, i64, i64, dp, i64, dp, i64, ctypes.POINTER(i64)]),
        "or_backward": (None, [i64, i64, cdp, i64, cdp, i64, cdp, i64, cdp, i64, dp, i64]),
        "or_householder": (None, [i64, i64, cdp, i64, dp, i64, dp, i64]),
    }


def open_library(path: str):
    """Load an oracle shared library (the default build, or a test's own)."""
    lib = ctypes.CDLL(path)
    for name, (res, args) in _sigs().items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = open_library(build())
        return _lib


@contextlib.contextmanager
def using_library(lib):
    """Route the module's functions to another oracle build (mutation tests)."""
    global _lib
    _load()
    with _lock:
        old, _lib = _lib, lib
    try:
        yield
    finally:
        with _lock:
            _lib = old


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    """A column-major FP64 copy of `a` (the C routines work in place)."""
    return np.array(a, dtype=np.float64, order="F", copy=True)


class OracleError(RuntimeError):
    """Raised when a factorisation reports a Cholesky breakdown or bad argument."""

    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status}")
        self.status = status


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_block_rows(rows: int) -> None:
    _load().or_set_block_rows(int(rows))


def get_block_rows() -> int:
    return int(_load().or_get_block_rows())


def gram(X) -> np.ndarray:
    """W = X^T X (Alg. 1 step 1), symmetric, fixed-order row sums."""
    X = _f64(X)
    m, b = X.shape
    W = np.zeros((b, b), order="F")
    _load().or_gram(m, b, _p(X), max(m, 1), _p(W), b)
    return W


def tn(X, Z) -> np.ndarray:
    """Y = X^T Z (the projection of Alg. 6 step 6 / Alg. 9 step 3)."""
    X, Z = _f64(X), _f64(Z)
    m, p = X.shape
    q = Z.shape[1]
    Y = np.zeros((p, q), order="F")
    _load().or_tn(m, p, q, _p(X), max(m, 1), _p(Z), max(m, 1), _p(Y), max(p, 1))
    return Y


def chol(W):
    """(U, status): upper U with U^T U = W (Alg. 1 step 2); status j+1 on breakdown."""
    W = _f64(W)
    b = W.shape[0]
    U = np.zeros((b, b), order="F")
    st = _load().or_chol(b, _p(W), b, _p(U), b)
    return U, int(st)


def trsm(X, U) -> np.ndarray:
    """Q = X U^{-1} by forward substitution (Alg. 1 step 3)."""
    X, U = _f64(X), _f64(U)
    m, b = X.shape
    _load().or_trsm(m, b, _p(X), max(m, 1), _p(U), b)
    return X


def update(X, Q, Y) -> np.ndarray:
    """X - Q Y (Alg. 6 step 7, Alg. 9 steps 4 and 7)."""
    X, Q, Y = _f64(X), _f64(Q), _f64(Y)
    m, q = X.shape
    p = Q.shape[1]
    _load().or_update(m, p, q, _p(X), max(m, 1), _p(Q), max(m, 1), _p(Y), max(p, 1))
    return X


def _factor(fn, A, *extra, what=""):
    A = _f64(A)
    m, n = A.shape
    R = np.zeros((n, n), order="F")
    st = fn(m, n, *extra, _p(A), max(m, 1), _p(R), n)
    return A, R, int(st)


def cqr(A, check=True):
    """Alg. 1 (CholeskyQR). Returns (Q, R) or (Q, R, status) with check=False."""
    Q, R, st = _factor(_load().or_cqr, A)
    return _ret(Q, R, st, check, "cqr")


def scqr(A, check=True):
    """Alg. 4 (shifted CholeskyQR, s = sqrt(m) u ||A||_F^2)."""
    Q, R, st = _factor(_load().or_scqr, A)
    return _ret(Q, R, st, check, "scqr")


def cqr2(A, check=True):
    """Alg. 3 (CholeskyQR2)."""
    Q, R, st = _factor(_load().or_cqr2, A)
    return _ret(Q, R, st, check, "cqr2")


def scqr3(A, check=True):
    """Alg. 5 (shifted CholeskyQR3)."""
    Q, R, st = _factor(_load().or_scqr3, A)
    return _ret(Q, R, st, check, "scqr3")


def cqrgs(A, b, check=True):
    """Alg. 6 (CholeskyQR with block Gram-Schmidt), panel width b."""
    Q, R, st = _factor(_load().or_cqrgs, A, int(b))
    return _ret(Q, R, st, check, "cqrgs")


def cqr2gs(A, b, check=True):
    """Alg. 7 (CholeskyQR2 with Gram-Schmidt), panel width b."""
    Q, R, st = _factor(_load().or_cqr2gs, A, int(b))
    return _ret(Q, R, st, check, "cqr2gs")


def mcqr2gs(A, b, check=True, literal_r=False, adaptive=False, inplace=False):
    """Alg. 9 (modified CholeskyQR2 with Gram-Schmidt), panel width b.
    adaptive=True: the runtime choice of the second CholeskyQR pass (Sec. 7).
    inplace=True: A must be a Fortran-ordered float64 array; it is
    overwritten by Q instead of copied first (for matrices of tens of GB)."""
    lib = _load()
    if inplace:
        if not (isinstance(A, np.ndarray) and A.dtype == np.float64 and A.flags.f_contiguous):
            raise ValueError("inplace=True needs a Fortran-ordered float64 array")
    else:
        A = _f64(A)
    m, n = A.shape
    R = np.zeros((n, n), order="F")
    flags = (LITERAL_R if literal_r else 0) | (ADAPTIVE if adaptive else 0)
    st = lib.or_mcqr2gs(m, n, int(b), _p(A), max(m, 1), _p(R), n, flags)
    return _ret(A, R, int(st), check, "mcqr2gs")


def mcqr2gs_halving(A, b, check=True):
    """Alg. 9 with the adaptive panel width: a panel whose first CholeskyQR
    breaks down or has (max U_ii / min U_ii)^2 > 1/(64 u) is retried with the
    largest divisor of b that is <= b/2, and later panels keep that width.
    Returns (Q, R, b_final), or (Q, R, b_final, status) with check=False."""
    lib = _load()
    A = _f64(A)
    m, n = A.shape
    R = np.zeros((n, n), order="F")
    bf = ctypes.c_int64(0)
    st = int(lib.or_mcqr2gs_halving(m, n, int(b), _p(A), max(m, 1), _p(R), n, ctypes.byref(bf)))
    if check:
        if st != 0:
            raise OracleError(st, "mcqr2gs_halving")
        return A, R, int(bf.value)
    return A, R, int(bf.value), st


def _ret(Q, R, st, check, what):
    if check:
        if st != 0:
            raise OracleError(st, what)
        return Q, R
    return Q, R, st


def backward(Q, R, dQ, dR) -> np.ndarray:
    """Abar for A = QR: M = R Rbar^T - Qbar^T Q; Abar = (Qbar + Q copyltu(M)) R^{-T}."""
    Q, R, dQ, dR = _f64(Q), _f64(R), _f64(dQ), _f64(dR)
    m, n = Q.shape
    dA = np.zeros((m, n), order="F")
    _load().or_backward(m, n, _p(Q), max(m, 1), _p(R), n, _p(dQ), max(m, 1), _p(dR), n, _p(dA), max(m, 1))
    return dA


def householder(A):
    """Textbook Householder QR, sign-normalised to diag(R) >= 0 (test pin only)."""
    A = _f64(A)
    m, n = A.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    _load().or_householder(m, n, _p(A), max(m, 1), _p(Q), max(m, 1), _p(R), n)
    return Q, R


FACTOR = {
    "mcqr2gs": lambda A, b, check=True: mcqr2gs(A, b, check=check),
    "cqr2gs": lambda A, b, check=True: cqr2gs(A, b, check=check),
    "cqr2": lambda A, b=None, check=True: cqr2(A, check=check),
}


if __name__ == "__main__":  # pragma: no cover - manual build entry
    print(build(force="--force" in sys.argv))
