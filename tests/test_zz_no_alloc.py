"""cqr_factor_noalloc: the factorisation for callers that cannot allocate
device memory when they factor (a memory budget fixed at start-up, a call
made from inside another allocator or memory pool, a no-allocation-after-
initialisation rule).  Its scratch is a fixed device array inside the
library instead of a caller workspace.

Called through the C ABI and checked against cqr_factor (the entry point
with a caller workspace) on two calls in a row, with the tolerances of the
parity tests.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from _helpers import orth_err, rel_diff, resid
from testmatrices import make_test_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R_TOL, Q_TOL, ORTH_TOL, RES_TOL = 1e-11, 1e-11, 1e-13, 1e-14


def _noalloc(P, A, b, variant):
    L = P.load()
    m, n = A.shape
    Q = P.empty_colmajor(m, n, "cuda")
    R = P.empty_colmajor(n, n, "cuda")
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    rc = L.cqr_factor_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), A.stride(1), b, ctypes.c_void_p(Q.data_ptr()),
                              Q.stride(1), ctypes.c_void_p(R.data_ptr()), R.stride(1), P.VARIANTS[variant],
                              ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    assert rc == 0, P.status_string(rc)
    torch.cuda.synchronize()
    return Q, R, int(status.item())


def test_noalloc_matches_workspace_entry_point_twice(cuda_lib):
    P = cuda_lib
    cases = [(30011, 64, 16, 1e10, 3001, "mcqr2gs"), (20000, 128, 32, 1e5, 3002, "cqr2gs")]
    for m, n, b, kappa, seed, variant in cases:  # two calls in a row, different sizes
        A = make_test_matrix(m, n, kappa, seed)
        At = P.colmajor(torch.from_numpy(A).cuda())
        Qn, Rn, st = _noalloc(P, At, b, variant)
        assert st == 0
        Qw, Rw = P.factor(At, b, variant)
        Qn, Rn, Qw, Rw = (x.cpu().numpy() for x in (Qn, Rn, Qw, Rw))
        assert rel_diff(Rn, Rw) <= R_TOL
        assert np.abs(Qn - Qw).max() <= Q_TOL
        assert orth_err(Qn) <= ORTH_TOL and resid(A, Qn, Rn) <= RES_TOL


def test_noalloc_reports_breakdown_and_rejects_oversize(cuda_lib):
    P = cuda_lib
    A = make_test_matrix(5000, 16, 1e3, seed=3003)
    A[:, 5] = 0.0
    _, _, st = _noalloc(P, P.colmajor(torch.from_numpy(A).cuda()), 4, "mcqr2gs")
    assert st == 6
    # a factorisation whose scratch exceeds the fixed array is refused, nothing launched
    L = P.load()
    m, n, b = 16384, 16384, 512  # the re-orthogonalisation coefficients Z alone need n*b*8 = 64 MiB
    assert P.workspace_size(m, n, b, "mcqr2gs") > P._capi.NOALLOC_SCRATCH_BYTES
    Z = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(Z.data_ptr())
    rc = L.cqr_factor_noalloc(m, n, p, m, b, p, m, p, n, P.VARIANTS["mcqr2gs"], None,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == P._capi.ERR_NOALLOC_TOO_LARGE
