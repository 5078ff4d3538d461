"""GB300-native FP64 CholeskyQR library (arXiv 2405.04237).

QR factorisation A = Q R of tall-and-skinny FP64 matrices by the modified
CholeskyQR2 with block Gram-Schmidt (mCQR2GS, Alg. 9), CQR2GS (Alg. 7),
CholeskyQR2 (Alg. 3) and shifted CholeskyQR3 (Alg. 5), with a hand-written
adjoint, a batched path and a panel-width autotuner.

The compute runs in the CUDA library behind the C ABI of ``include/cqr.h``;
this module only marshals torch tensors (device memory, the current stream)
into that ABI.  There is no CPU fallback.

Layout: the library is column-major.  A torch matrix with strides (1, ld) is
passed as is; any other layout is copied to a column-major buffer first.
Outputs are returned as column-major tensors (strides (1, m) and (1, n)).
"""
from __future__ import annotations

import ctypes

import torch

from . import _capi
from ._capi import CQRError, VARIANTS, load, status_string

__all__ = [
    "factor", "qr", "backward", "factor_batched", "workspace_size", "default_panel",
    "CQRFunction", "CQRError", "read_status", "probe_fp64_peak", "probe_fp64", "colmajor", "empty_colmajor",
    "launch_count", "KernelTimer", "BatchedGraph", "batched_workspace_size", "qr_batched", "CQRBatchedFunction",
    "use_torch_allocator", "read_panel_width", "batched_panel_widths", "factor_host", "empty_colmajor_pinned", "PhaseTrace",
]


def _variant(v) -> int:
    if isinstance(v, str):
        return VARIANTS[v.lower()]
    return int(v)


def colmajor(A: torch.Tensor) -> torch.Tensor:
    """A column-major view of A if it already is one, else a column-major copy."""
    if A.dim() != 2:
        raise ValueError("expected a matrix")
    m, n = A.shape
    if A.stride(0) == 1 and (n <= 1 or A.stride(1) >= max(m, 1)):
        return A
    return A.t().contiguous().t()


def empty_colmajor(m: int, n: int, device, dtype=torch.float64) -> torch.Tensor:
    return torch.empty((n, m), dtype=dtype, device=device).t()


def _ld(A: torch.Tensor) -> int:
    m, n = A.shape
    return max(A.stride(1) if n > 1 else m, m, 1)


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_input(A: torch.Tensor):
    if not A.is_cuda:
        raise ValueError("inputs must be CUDA tensors (the library has no CPU path)")
    if A.dtype != torch.float64:
        raise ValueError("inputs must be float64")
    if A.dim() != 2:
        raise ValueError("inputs must be matrices")


_torch_alloc_callbacks = None


def use_torch_allocator(enable: bool = True) -> None:
    """Register torch's CUDA caching allocator with cqr_set_allocator, for C
    calls made with workspace = NULL (those calls synchronise their stream
    before they free, so the caching allocator may reuse the block at once).
    enable=False unregisters it."""
    global _torch_alloc_callbacks
    L = load()
    if not enable:
        rc = L.cqr_set_allocator(_capi.ALLOC_FN(), _capi.FREE_FN(), None)
        _torch_alloc_callbacks = None
        if rc != 0:
            raise CQRError(rc, "cqr_set_allocator")
        return

    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          int(stream or 0)))
        except Exception:  # the library sees NULL and returns CQR_ERR_ALLOC
            return None

    def _free(ptr, nbytes, stream, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    cbs = (_capi.ALLOC_FN(_alloc), _capi.FREE_FN(_free))
    rc = L.cqr_set_allocator(cbs[0], cbs[1], None)
    if rc != 0:
        raise CQRError(rc, "cqr_set_allocator")
    _torch_alloc_callbacks = cbs  # keep the ctypes thunks alive while registered


def default_panel(n: int) -> int:
    return int(load().cqr_default_panel(int(n)))


def workspace_size(m: int, n: int, panel_b: int = 0, variant="mcqr2gs", emulated: bool = False,
                   halving: bool = False) -> int:
    return int(load().cqr_workspace_size(int(m), int(n), int(panel_b), _variant(variant) | (
        _capi.EMULATED if emulated else 0) | (_capi.HALVE if halving else 0)))


def _batch_flags(variant, schedule="auto", group=0, halving=False) -> int:
    if schedule not in ("auto", "pool"):
        raise ValueError("schedule must be 'auto' (persistent launch where eligible) or 'pool'")
    return (_variant(variant) | (_capi.BATCH_POOL if schedule == "pool" else 0) | _capi.BATCH_GROUP(group)
            | (_capi.HALVE if halving else 0))


def batched_workspace_size(ms, ns, panel_b, variant="mcqr2gs", schedule="auto", group=0, halving=False) -> int:
    B = len(ms)
    return int(load().cqr_batched_workspace_size(B, (ctypes.c_int64 * B)(*ms), (ctypes.c_int64 * B)(*ns),
                                                 (ctypes.c_int * B)(*[int(b) for b in panel_b]),
                                                 _batch_flags(variant, schedule, group, halving)))


def batched_panel_widths(workspace: torch.Tensor, batch: int, stream=None) -> list:
    """Final panel width of each matrix of the last persistent batched call that used `workspace`."""
    out = (ctypes.c_int * int(batch))()
    rc = load().cqr_batched_panel_widths(int(batch), _ptr(workspace), _stream(stream), out)
    if rc != 0:
        raise CQRError(rc, "cqr_batched_panel_widths")
    return list(out)


def read_panel_width(workspace: torch.Tensor, stream=None) -> int:
    """Width of the last panel of the last halving=True factorisation that used `workspace`."""
    b = ctypes.c_int(0)
    rc = load().cqr_read_panel_width(_ptr(workspace), _stream(stream), ctypes.byref(b))
    if rc != 0:
        raise CQRError(rc, "cqr_read_panel_width")
    return int(b.value)


def read_status(workspace: torch.Tensor, stream=None) -> int:
    st = ctypes.c_int(0)
    rc = load().cqr_read_status(_ptr(workspace), _stream(stream), ctypes.byref(st))
    if rc != 0:
        raise CQRError(rc, "cqr_read_status")
    return int(st.value)


def factor(A: torch.Tensor, panel_b: int = 0, variant="mcqr2gs", *, inplace: bool = False, check: bool = True,
           out=None, workspace: torch.Tensor | None = None, stream=None, lookahead: bool = False,
           adaptive: bool = False, emulated: bool = False, halving: bool = False, info: dict | None = None):
    """A = Q R.  Returns (Q, R) as column-major FP64 tensors.

    inplace=True overwrites A's (column-major) storage with Q.  lookahead=True
    overlaps each trailing update with the next panel's CholeskyQR on a side
    stream (bitwise-identical results).  adaptive=True (mCQR2GS) applies the
    runtime choice of the second CholeskyQR pass per panel.  emulated=True
    (mCQR2GS) runs the m-row products (Gram matrices, projections, updates)
    on the FP8 tensor cores with the FP64-accurate Ozaki splitting.
    halving=True (mCQR2GS) applies the adaptive panel width: a panel whose
    first CholeskyQR breaks down or is too ill-conditioned is retried with a
    halved width (synchronous; the final width goes to info["panel_b"] when
    a dict is given).  check=True
    synchronises the stream and raises CQRError on a Cholesky breakdown; with
    check=False the call is fully asynchronous (and graph-capturable when a
    workspace and outputs are supplied).
    """
    _check_input(A)
    L = load()
    m, n = A.shape
    var = _variant(variant)
    Ac = colmajor(A)
    if inplace and Ac.data_ptr() != A.data_ptr():
        raise ValueError("inplace=True needs a column-major A")
    if out is not None:
        Q, R = out
    else:
        Q = Ac if inplace else empty_colmajor(m, n, A.device)
        R = empty_colmajor(n, n, A.device)
    flags = var | (_capi.LOOKAHEAD if lookahead else 0) | (_capi.ADAPTIVE if adaptive else 0) | (
        _capi.EMULATED if emulated else 0) | (_capi.HALVE if halving else 0)
    ws_bytes = L.cqr_workspace_size(m, n, int(panel_b), flags)
    if ws_bytes == 0:
        raise CQRError(-5 if n > 0 and m >= n else -1, "cqr_workspace_size")
    if workspace is None:
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=A.device)
    elif workspace.numel() < ws_bytes:
        raise ValueError(f"workspace too small: {workspace.numel()} < {ws_bytes}")
    st = _stream(stream)
    rc = L.cqr_factor(m, n, _ptr(Ac), _ld(Ac), int(panel_b), _ptr(Q), _ld(Q), _ptr(R), _ld(R), flags,
                      _ptr(workspace), ctypes.c_size_t(workspace.numel()), st)
    if rc != 0:
        raise CQRError(rc, "cqr_factor")
    if halving and info is not None:
        info["panel_b"] = read_panel_width(workspace, stream)
    if check:
        s = read_status(workspace, stream)
        if s != 0:
            raise CQRError(s, "cqr_factor")
    return Q, R


def empty_colmajor_pinned(m: int, n: int) -> torch.Tensor:
    """A page-locked host m x n column-major FP64 matrix (for factor_host)."""
    return torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()


def factor_host(A: torch.Tensor, panel_b: int = 0, variant="mcqr2gs", *, out=None, device_out=None,
                workspace: torch.Tensor | None = None, stream=None, lookahead: bool = False, adaptive: bool = False,
                emulated: bool = False, halving: bool = False, check: bool = True, info: dict | None = None,
                device=None):
    """A = Q R for a HOST matrix A (CPU float64, column-major; page-locked
    for the copy overlap).  The library copies A to the device buffer Qd,
    factors it there and copies Q and R back, the copies overlapped with the
    factorisation (cqr_factor_host).  out=(Q, R): host outputs (default: new
    page-locked column-major matrices; Q may be A itself).  device_out=(Qd,
    Rd): the CUDA buffers the factorisation runs in (default: new ones on
    `device`, else the current device).  The remaining options are factor()'s.
    Returns the host (Q, R); with check=False the call is asynchronous and
    they are complete once `stream` is."""
    if A.is_cuda or A.dtype != torch.float64 or A.dim() != 2:
        raise ValueError("factor_host takes a CPU float64 matrix")
    L = load()
    m, n = A.shape
    Ac = colmajor(A)
    if out is not None:
        Q, R = out
    else:
        Q, R = empty_colmajor_pinned(m, n), empty_colmajor_pinned(n, n)
    for t in (Q, R):
        if t.is_cuda or t.dtype != torch.float64 or colmajor(t).data_ptr() != t.data_ptr():
            raise ValueError("host outputs must be column-major CPU float64 matrices")
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if device_out is not None:
        Qd, Rd = device_out
    else:
        Qd, Rd = empty_colmajor(m, n, dev), empty_colmajor(n, n, dev)
    for t in (Qd, Rd):
        _check_input(t)
        if colmajor(t).data_ptr() != t.data_ptr():
            raise ValueError("device buffers must be column-major")
    flags = _variant(variant) | (_capi.LOOKAHEAD if lookahead else 0) | (_capi.ADAPTIVE if adaptive else 0) | (
        _capi.EMULATED if emulated else 0) | (_capi.HALVE if halving else 0)
    ws_bytes = L.cqr_workspace_size(m, n, int(panel_b), flags)
    if ws_bytes == 0:
        raise CQRError(-5 if n > 0 and m >= n else -1, "cqr_workspace_size")
    if workspace is None:
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=Qd.device)
    elif workspace.numel() < ws_bytes:
        raise ValueError(f"workspace too small: {workspace.numel()} < {ws_bytes}")
    st = _stream(stream)
    rc = L.cqr_factor_host(m, n, _ptr(Ac), _ld(Ac), int(panel_b), _ptr(Q), _ld(Q), _ptr(R), _ld(R), flags,
                           _ptr(Qd), _ld(Qd), _ptr(Rd), _ld(Rd), _ptr(workspace),
                           ctypes.c_size_t(workspace.numel()), st)
    if rc != 0:
        raise CQRError(rc, "cqr_factor_host")
    if halving and info is not None:
        info["panel_b"] = read_panel_width(workspace, stream)
    if check:
        s = read_status(workspace, stream)
        if s != 0:
            raise CQRError(s, "cqr_factor_host")
    return Q, R


def backward(Q: torch.Tensor, R: torch.Tensor, dQ: torch.Tensor | None, dR: torch.Tensor | None, stream=None):
    """Abar for A = QR: M = R Rbar^T - Qbar^T Q; Abar = (Qbar + Q copyltu(M)) R^{-T}."""
    for t in (Q, R, dQ, dR):
        if t is not None:
            _check_input(t)
    if R.shape != (Q.shape[1], Q.shape[1]) or (dQ is not None and dQ.shape != Q.shape) or (
            dR is not None and dR.shape != R.shape):
        raise ValueError("backward: Q (m x n), R (n x n), dQ like Q, dR like R")
    L = load()
    m, n = Q.shape
    Qc, Rc = colmajor(Q), colmajor(R)
    dQc = colmajor(dQ) if dQ is not None else None
    dRc = colmajor(dR) if dR is not None else None
    dA = empty_colmajor(m, n, Q.device)
    ws_bytes = L.cqr_backward_workspace_size(m, n)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=Q.device)
    rc = L.cqr_backward(m, n, _ptr(Qc), _ld(Qc), _ptr(Rc), _ld(Rc), _ptr(dQc), _ld(dQc) if dQc is not None else m,
                        _ptr(dRc), _ld(dRc) if dRc is not None else n, _ptr(dA), _ld(dA), _ptr(ws),
                        ctypes.c_size_t(ws.numel()), _stream(stream))
    if rc != 0:
        raise CQRError(rc, "cqr_backward")
    return dA


class CQRFunction(torch.autograd.Function):
    """Differentiable A -> (Q, R).  Saves only the outputs (Q, R): the adjoint
    needs no per-panel intermediates, so nothing else is kept between the
    forward and backward passes."""

    @staticmethod
    def forward(ctx, A, panel_b=0, variant="mcqr2gs"):
        Q, R = factor(A.detach(), panel_b, variant)
        ctx.save_for_backward(Q, R)
        return Q, R

    @staticmethod
    def backward(ctx, dQ, dR):
        Q, R = ctx.saved_tensors
        return backward(Q, R, dQ, dR), None, None


def qr(A: torch.Tensor, panel_b: int = 0, variant="mcqr2gs"):
    """Differentiable QR (see CQRFunction)."""
    return CQRFunction.apply(A, panel_b, variant)


def factor_batched(As, panel_b=None, variant="mcqr2gs", *, check: bool = True, stream=None, workspace=None,
                   status=None, inplace: bool = False, schedule: str = "auto", group: int = 0,
                   halving: bool = False):
    """Factor a list of column-major FP64 CUDA matrices in one batched call.

    Returns a list of (Q_i, R_i).  schedule="auto" runs mCQR2GS batches of
    matrices with n <= 128 (n, b multiples of 4) as one persistent launch
    (groups of `group` CTAs per matrix, 0 = library default; halving=True
    narrows rejected panels on the device) -- equal to factor(A_i, b_i) to
    rounding; otherwise, or with schedule="pool", each result is bitwise
    factor(A_i, b_i).
    """
    L = load()
    B = len(As)
    if B == 0:
        return []
    var = _variant(variant)
    dev = As[0].device
    Acs = [colmajor(A) for A in As]
    for A in Acs:
        _check_input(A)
    if inplace and any(Ac.data_ptr() != A.data_ptr() for Ac, A in zip(Acs, As)):
        raise ValueError("inplace=True needs column-major inputs")
    ms = (ctypes.c_int64 * B)(*[A.shape[0] for A in Acs])
    ns = (ctypes.c_int64 * B)(*[A.shape[1] for A in Acs])
    lds = (ctypes.c_int64 * B)(*[_ld(A) for A in Acs])
    if panel_b is None:
        panel_b = [0] * B
    elif isinstance(panel_b, int):
        panel_b = [panel_b] * B
    bs = (ctypes.c_int * B)(*[int(b) for b in panel_b])
    Qs = [A if inplace else empty_colmajor(A.shape[0], A.shape[1], dev) for A in Acs]
    Rs = [empty_colmajor(A.shape[1], A.shape[1], dev) for A in Acs]
    # Q_i must share A_i's leading dimension (ldq_i = lda_i)
    for i, (A, Q) in enumerate(zip(Acs, Qs)):
        if _ld(Q) != _ld(A):
            Qs[i] = torch.empty((A.shape[1], _ld(A)), dtype=torch.float64, device=dev).t()[: A.shape[0]]
    Ap = (ctypes.c_void_p * B)(*[A.data_ptr() for A in Acs])
    Qp = (ctypes.c_void_p * B)(*[Q.data_ptr() for Q in Qs])
    Rp = (ctypes.c_void_p * B)(*[R.data_ptr() for R in Rs])
    flags = _batch_flags(var, schedule, group, halving)
    ws_bytes = L.cqr_batched_workspace_size(B, ms, ns, bs, flags)
    if ws_bytes == 0:
        raise CQRError(-2, "cqr_batched_workspace_size")
    if workspace is None:
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    if status is None:
        status = torch.zeros(B, dtype=torch.int32, device=dev)
    rc = L.cqr_factor_batched(B, ms, ns, lds, bs, Ap, Qp, Rp, flags, _ptr(status), _ptr(workspace),
                              ctypes.c_size_t(workspace.numel()), _stream(stream))
    if rc != 0:
        raise CQRError(rc, "cqr_factor_batched")
    if check:
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        bad = torch.nonzero(status).flatten().tolist()
        if bad:
            raise CQRError(int(status[bad[0]].item()), f"cqr_factor_batched (matrix {bad[0]})")
    return list(zip(Qs, Rs))


class CQRBatchedFunction(torch.autograd.Function):
    """Differentiable A_i -> (Q_i, R_i) for a list of matrices: one batched
    forward call (cqr_factor_batched, persistent launch where eligible), one
    adjoint call (cqr_backward) per matrix in the backward pass.  Saves only
    the outputs; each gradient is bitwise backward(Q_i, R_i, Qbar_i, Rbar_i)."""

    @staticmethod
    def forward(ctx, panel_b, variant, *As):
        outs = factor_batched([A.detach() for A in As], panel_b, variant)
        Qs = [Q for Q, _ in outs]
        Rs = [R for _, R in outs]
        ctx.save_for_backward(*Qs, *Rs)
        ctx.count = len(As)
        return (*Qs, *Rs)

    @staticmethod
    def backward(ctx, *grads):
        B = ctx.count
        saved = ctx.saved_tensors
        dAs = [backward(saved[i], saved[B + i], grads[i], grads[B + i]) for i in range(B)]
        return (None, None, *dAs)


def qr_batched(As, panel_b=None, variant="mcqr2gs"):
    """Differentiable batched QR (see CQRBatchedFunction); returns a list of
    (Q_i, R_i).  panel_b: one width for all, a list, or None (library default)."""
    if len(As) == 0:
        return []
    out = CQRBatchedFunction.apply(panel_b, variant, *As)
    B = len(As)
    return list(zip(out[:B], out[B:]))


class BatchedGraph:
    """A batched factorisation captured once into a CUDA graph and replayed.

    Inputs are the given column-major matrices (their storage is read on every
    replay, so refill them in place to factor new data); outputs Q_i, R_i and
    the per-matrix status live in buffers owned by this object.  The first
    (eager) call checks every status; capture happens after it.
    """

    def __init__(self, As, panel_b=None, variant="mcqr2gs", schedule="auto", group=0, halving=False):
        self.As = [colmajor(A) for A in As]
        self.panel_b = panel_b
        self.variant = variant
        self.flags = _batch_flags(variant, schedule, group, halving)
        dev = self.As[0].device
        L = load()
        B = len(self.As)
        bs = self._panels()
        ms = (ctypes.c_int64 * B)(*[A.shape[0] for A in self.As])
        ns = (ctypes.c_int64 * B)(*[A.shape[1] for A in self.As])
        self.workspace = torch.empty(batched_workspace_size(list(ms), list(ns), list(bs), variant, schedule, group,
                                                            halving), dtype=torch.uint8, device=dev)
        self.status = torch.zeros(B, dtype=torch.int32, device=dev)
        self.out = factor_batched(self.As, list(bs), variant, workspace=self.workspace, status=self.status,
                                  schedule=schedule, group=group, halving=halving)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._launch()

    def _panels(self):
        B = len(self.As)
        pb = self.panel_b if self.panel_b is not None else [0] * B
        if isinstance(pb, int):
            pb = [pb] * B
        return (ctypes.c_int * B)(*[int(b) for b in pb])

    def _launch(self):
        L = load()
        B = len(self.As)
        ms = (ctypes.c_int64 * B)(*[A.shape[0] for A in self.As])
        ns = (ctypes.c_int64 * B)(*[A.shape[1] for A in self.As])
        lds = (ctypes.c_int64 * B)(*[_ld(A) for A in self.As])
        Ap = (ctypes.c_void_p * B)(*[A.data_ptr() for A in self.As])
        Qp = (ctypes.c_void_p * B)(*[Q.data_ptr() for Q, _ in self.out])
        Rp = (ctypes.c_void_p * B)(*[R.data_ptr() for _, R in self.out])
        rc = L.cqr_factor_batched(B, ms, ns, lds, self._panels(), Ap, Qp, Rp, self.flags,
                                  _ptr(self.status), _ptr(self.workspace), ctypes.c_size_t(self.workspace.numel()),
                                  _stream(None))
        if rc != 0:
            raise CQRError(rc, "cqr_factor_batched")

    def replay(self):
        self.graph.replay()
        return self.out


def probe_fp64_peak(iters: int = 20000) -> float:
    """Measured FP64 FMA throughput of the current GPU, GFLOP/s."""
    return float(load().cqr_probe_fp64_peak(int(iters)))


PROBE_KINDS = {"dfma": 0, "dmma_m8n8k4": 1, "dmma_m16n8k16": 2}


def probe_fp64(kind: str = "dfma", iters: int = 100000) -> dict:
    """FP64 peak microbenchmark (cqr_probe_fp64): GFLOP/s, flop per clock per
    SM (from the SM cycle counters) and the effective SM clock in MHz."""
    g, f, c = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    rc = load().cqr_probe_fp64(PROBE_KINDS[kind], int(iters), ctypes.byref(g), ctypes.byref(f), ctypes.byref(c))
    if rc != 0:
        raise CQRError(rc, "cqr_probe_fp64")
    return {"kind": kind, "gflops": g.value, "flop_per_clk_sm": f.value, "sm_mhz": c.value}


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load().cqr_launch_count())


class PhaseTrace:
    """Context manager: records the phase ranges the library brackets its
    enqueue with (the same ranges it emits as NVTX, domain "cqr") as
    (phase, panel, begin) tuples in ``.events``, through cqr_set_trace."""

    def __init__(self):
        self.events = []
        self._cb = None

    def __enter__(self):
        def _cb(name, panel, begin, ctx):
            self.events.append((name.decode(), int(panel), int(begin)))

        self._cb = _capi.TRACE_FN(_cb)
        load().cqr_set_trace(self._cb, None)
        return self

    def __exit__(self, *exc):
        load().cqr_set_trace(_capi.TRACE_FN(), None)
        self._cb = None
        return False

    def phases(self):
        """The (phase, panel) pairs in the order they began."""
        return [(n, p) for n, p, b in self.events if b]


class KernelTimer:
    """Context manager: times every library kernel launch inside it with CUDA
    events on its own stream; ``.read()`` gives per-class launches, device ms
    and algorithmic FLOPs."""

    def __init__(self, capacity: int = 100000):
        self.capacity = int(capacity)

    def __enter__(self):
        rc = load().cqr_profile_enable(self.capacity)
        if rc != 0:
            raise CQRError(rc, "cqr_profile_enable")
        return self

    def __exit__(self, *exc):
        load().cqr_profile_disable()
        return False

    def read(self) -> dict:
        out = {}
        L = load()
        for cls, name in enumerate(_capi.KERNEL_CLASSES):
            n, ms, fl = ctypes.c_longlong(0), ctypes.c_double(0), ctypes.c_double(0)
            rc = L.cqr_profile_read(cls, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl))
            if rc != 0:
                raise CQRError(rc, "cqr_profile_read")
            out[name] = {"launches": int(n.value), "ms": float(ms.value), "flops": float(fl.value)}
        return out
