"""Failure detection on the GPU: a bounded wait that expires.

Every mbarrier wait inside the tensor-core kernels of the emulated variant
is bounded in time.  The one-shot test hook cqr_test_arm_wait_expiry makes
the next launch of one kernel withhold the copies of one stage (nothing
completes the barrier those waits watch) with a 1 ms bound.  The test
checks, through the C ABI, that
  * the status word reads CQR_STATUS_TIMEOUT and the call returns (no hang,
    no fault: every later kernel of the call sees the status and returns);
  * the kernel freed its tensor memory and the context stays usable: the
    next emulated factorisation on the same context (which allocates tensor
    memory again in the same kernels) succeeds and meets the accuracy
    bounds, and so does a native one;
  * the hook disarmed itself after one launch.
Nothing here faults, traps or hangs the GPU: the withheld copies are never
issued, so the wait simply runs out.
"""
import ctypes

import numpy as np
import pytest

from _helpers import orth_err, resid
from testmatrices import make_test_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WAIT_NS = 1_000_000  # 1 ms


@pytest.mark.parametrize("kernel,stage", [(0, 1), (0, 0), (1, 0), (1, 1)])
def test_wait_expiry_reports_timeout_and_context_survives(cuda_lib, kernel, stage):
    P = cuda_lib
    L = P.load()
    m, n, b = 20000, 256, 64
    A = make_test_matrix(m, n, 1e8, seed=6100 + kernel)
    At = P.colmajor(torch.from_numpy(A).cuda())
    Q, R = P.empty_colmajor(m, n, "cuda"), P.empty_colmajor(n, n, "cuda")
    ws = torch.empty(P.workspace_size(m, n, b, "mcqr2gs", emulated=True), dtype=torch.uint8, device="cuda")
    assert L.cqr_test_arm_wait_expiry(kernel, stage, WAIT_NS) == 0
    try:
        P.factor(At, b, "mcqr2gs", out=(Q, R), workspace=ws, emulated=True, check=False)
        assert P.read_status(ws) == P._capi.STATUS_TIMEOUT
    finally:
        L.cqr_test_arm_wait_expiry(-1, 0, 1)
    # the same context: emulated (tensor memory allocated again) and native factorisations succeed
    Qe, Re = P.factor(At, b, "mcqr2gs", out=(Q, R), workspace=ws, emulated=True)
    assert P.read_status(ws) == 0
    Qn, Rn = Qe.cpu().numpy(), Re.cpu().numpy()
    assert orth_err(Qn) <= 1e-13 and resid(A, Qn, Rn) <= 1e-14
    Qd, Rd = P.factor(At, b, "mcqr2gs")
    assert orth_err(Qd.cpu().numpy()) <= 1e-13


def test_status_string_of_timeout(cuda_lib):
    assert "bounded wait" in cuda_lib.status_string(cuda_lib._capi.STATUS_TIMEOUT)
