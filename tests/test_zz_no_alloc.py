"""cqr_factor_noalloc: the factorisation for callers that cannot allocate
device memory when they factor (a memory budget fixed at start-up, a call
made from inside another allocator or memory pool, a no-allocation-after-
initialisation rule).  Its scratch is a fixed device array inside the
library instead of a caller workspace.

Called through the C ABI and checked against cqr_factor (the entry point
with a caller workspace) on two calls in a row.  Both entry points enqueue
the same kernel sequence with the same sizes, so the results must be equal
bit for bit; the norms are checked against the parity tests' bounds as
well.  A repeated call must leave the device's free memory unchanged (the
first call on a device may create the array).  The file name makes pytest
collect it last.
"""
import ctypes

import numpy as np
import pytest

from _helpers import orth_err, resid
from testmatrices import make_test_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORTH_TOL, RES_TOL = 1e-13, 1e-14


def _noalloc(P, A, b, variant, Q, R, status):
    L = P.load()
    m, n = A.shape
    s = torch.cuda.current_stream()
    rc = L.cqr_factor_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), A.stride(1), b, ctypes.c_void_p(Q.data_ptr()),
                              Q.stride(1), ctypes.c_void_p(R.data_ptr()), R.stride(1), P.VARIANTS[variant],
                              ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    assert rc == 0, P.status_string(rc)


def test_noalloc_matches_workspace_entry_point_twice(cuda_lib):
    P = cuda_lib
    cases = [(30011, 64, 16, 1e10, 3001, "mcqr2gs"), (20000, 128, 32, 1e5, 3002, "cqr2gs")]
    for m, n, b, kappa, seed, variant in cases:  # two sizes, each factored twice in a row
        A = make_test_matrix(m, n, kappa, seed)
        At = P.colmajor(torch.from_numpy(A).cuda())
        outs = [(P.empty_colmajor(m, n, "cuda"), P.empty_colmajor(n, n, "cuda"),
                 torch.full((1,), -7, dtype=torch.int32, device="cuda")) for _ in range(2)]
        _noalloc(P, At, b, variant, *outs[0])
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        _noalloc(P, At, b, variant, *outs[1])
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
        Qw, Rw = P.factor(At, b, variant)
        for Qn, Rn, st in outs:
            assert int(st.item()) == 0
            assert torch.equal(Qn, Qw) and torch.equal(Rn, Rw)
        Qn, Rn = outs[1][0].cpu().numpy(), outs[1][1].cpu().numpy()
        assert orth_err(Qn) <= ORTH_TOL and resid(A, Qn, Rn) <= RES_TOL


def test_noalloc_reports_breakdown_and_rejects_oversize(cuda_lib):
    P = cuda_lib
    A = make_test_matrix(5000, 16, 1e3, seed=3003)
    A[:, 5] = 0.0
    At = P.colmajor(torch.from_numpy(A).cuda())
    Q, R = P.empty_colmajor(5000, 16, "cuda"), P.empty_colmajor(16, 16, "cuda")
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    _noalloc(P, At, 4, "mcqr2gs", Q, R, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 6
    L = P.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    Z = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(Z.data_ptr())
    # variant flags are refused (argument 10)
    rc = L.cqr_factor_noalloc(5000, 16, ctypes.c_void_p(At.data_ptr()), 5000, 4, ctypes.c_void_p(Q.data_ptr()), 5000,
                              ctypes.c_void_p(R.data_ptr()), 16, P.VARIANTS["mcqr2gs"] | P._capi.LOOKAHEAD, None, s)
    assert rc == -10
    # a factorisation whose scratch exceeds the fixed array is refused, nothing launched
    m, n, b = 16384, 16384, 512  # the re-orthogonalisation coefficients Z alone need n*b*8 = 64 MiB
    assert P.workspace_size(m, n, b, "mcqr2gs") > P._capi.NOALLOC_SCRATCH_BYTES
    rc = L.cqr_factor_noalloc(m, n, p, m, b, p, m, p, n, P.VARIANTS["mcqr2gs"], None, s)
    assert rc == P._capi.ERR_NOALLOC_TOO_LARGE
