"""cqr_factor_host: A, Q and R in host memory, copies overlapped with the
factorisation.

The entry point runs the kernels of cqr_factor with the same arguments in
the same order (only the copies are added and interleaved), so its results
must equal, bit for bit, those of the device call on a copy of the same
matrix -- with every flag, every variant, padded leading dimensions, an
in-place host factorisation, pageable host buffers and a single-panel
matrix.  One case is also compared with the oracle element by element.
"""
import numpy as np
import pytest

from _helpers import orth_err, rel_diff, resid
from testmatrices import make_test_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def host_colmajor(A: np.ndarray, pinned=True, ld=None):
    m, n = A.shape
    ld = m if ld is None else ld
    buf = torch.empty((n, ld), dtype=torch.float64, pin_memory=pinned)
    buf[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T))
    return buf.t()[:m]


def device_ref(P, A, b, variant="mcqr2gs", **kw):
    At = P.colmajor(torch.from_numpy(np.asfortranarray(A)).cuda())
    Q, R = P.factor(At, b, variant, **kw)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), R.cpu().numpy()


def host_call(P, A, b, variant="mcqr2gs", pinned=True, lda=None, ldq=None, **kw):
    Ah = host_colmajor(A, pinned, lda)
    Qh = host_colmajor(np.zeros_like(A), pinned, ldq)
    Rh = host_colmajor(np.zeros((A.shape[1], A.shape[1])), pinned)
    Q, R = P.factor_host(Ah, b, variant, out=(Qh, Rh), **kw)
    assert Q.data_ptr() == Qh.data_ptr() and R.data_ptr() == Rh.data_ptr()
    return Q.numpy().copy(), R.numpy().copy()


@pytest.mark.parametrize("m,n,b,kappa,seed,kw", [
    (20000, 96, 32, 1e8, 1, {}),
    (20011, 96, 32, 1e12, 2, {"lookahead": True}),
    (30000, 128, 32, 1e5, 3, {"adaptive": True}),
    (16384, 64, 16, 1e10, 4, {"emulated": True}),
    (5000, 64, 64, 1e13, 1, {"halving": True}),     # the first panel is narrowed to 32 columns
    (12000, 48, 48, 1e6, 5, {}),                    # one panel: no second copy, Q_0 out at the end
])
def test_host_equals_device_mcqr2gs(cuda_lib, m, n, b, kappa, seed, kw):
    P = cuda_lib
    A = make_test_matrix(m, n, kappa, seed=seed)
    Qd, Rd = device_ref(P, A, b, **kw)
    Qh, Rh = host_call(P, A, b, **kw)
    assert np.array_equal(Qh, Qd) and np.array_equal(Rh, Rd)
    assert orth_err(Qh) <= 1e-13 and resid(A, Qh, Rh) <= 1e-14


@pytest.mark.parametrize("variant,m,n,b", [("cqr2gs", 9000, 64, 16), ("cqr2", 9000, 64, 0),
                                            ("scqr3", 9000, 64, 0)])
def test_host_equals_device_other_variants(cuda_lib, variant, m, n, b):
    P = cuda_lib
    A = make_test_matrix(m, n, 1e5 if variant == "cqr2" else 1e9, seed=7)
    Qd, Rd = device_ref(P, A, b, variant)
    Qh, Rh = host_call(P, A, b, variant)
    assert np.array_equal(Qh, Qd) and np.array_equal(Rh, Rd)


def test_host_padded_pageable_and_in_place(cuda_lib):
    P = cuda_lib
    A = make_test_matrix(10007, 96, 1e11, seed=11)
    Qd, Rd = device_ref(P, A, 32)
    # padded leading dimensions of host A and host Q
    Qh, Rh = host_call(P, A, 32, lda=10011, ldq=10240)
    assert np.array_equal(Qh, Qd) and np.array_equal(Rh, Rd)
    # pageable host buffers: the copies are synchronous, the results the same
    Qh, Rh = host_call(P, A, 32, pinned=False)
    assert np.array_equal(Qh, Qd) and np.array_equal(Rh, Rd)
    # in place on the host: Q overwrites A's storage
    Ah = host_colmajor(A, True, 10016)
    Rh = host_colmajor(np.zeros((96, 96)), True)
    Q, R = P.factor_host(Ah, 32, out=(Ah, Rh))
    assert np.array_equal(Ah.numpy(), Qd) and np.array_equal(R.numpy(), Rd)


def test_host_device_buffers_hold_the_result(cuda_lib):
    """Qd and Rd are left holding Q and R; the call is asynchronous with
    check=False and complete once the stream is."""
    P = cuda_lib
    m, n, b = 40000, 128, 32
    A = make_test_matrix(m, n, 1e9, seed=3)
    Ah = host_colmajor(A)
    Qd = P.empty_colmajor(m, n, "cuda")
    Rd = P.empty_colmajor(n, n, "cuda")
    s = torch.cuda.Stream()
    Qh, Rh = P.factor_host(Ah, b, device_out=(Qd, Rd), stream=s, check=False)
    s.synchronize()
    Qr, Rr = device_ref(P, A, b)
    assert np.array_equal(Qh.numpy(), Qr) and np.array_equal(Rh.numpy(), Rr)
    assert np.array_equal(Qd.cpu().numpy(), Qr) and np.array_equal(Rd.cpu().numpy(), Rr)


def test_host_matches_the_oracle(cuda_lib, oracle):
    P = cuda_lib
    A = make_test_matrix(6000, 96, 1e5, seed=21)
    Qo, Ro = oracle.mcqr2gs(A, 32)
    Qh, Rh = host_call(P, A, 32)
    # the tolerances of the device parity tests (kappa <= 1e6: element-wise)
    assert rel_diff(Rh, Ro) <= 1e-11 and np.abs(Qh - Qo).max() <= 1e-11


def test_host_breakdown_status(cuda_lib):
    """A zero column breaks the Cholesky factorisation; the status word
    reports the column as for the device call."""
    P = cuda_lib
    A = make_test_matrix(4000, 32, 1e3, seed=2)
    A[:, 20] = 0.0
    with pytest.raises(P.CQRError) as e:
        host_call(P, A, 16)
    with pytest.raises(P.CQRError) as e2:
        device_ref(P, A, 16)
    assert e.value.code == e2.value.code == 21
