"""workspace = NULL through a caller-registered allocator (cqr_set_allocator).

torch's caching allocator is registered (use_torch_allocator); the three
entry points are called through the C ABI with a NULL workspace and must
give the same bits as the calls with an explicit workspace (the same kernel
sequence runs), return the status word synchronously (cqr_factor), and hand
every byte back (torch's allocated-memory counter is unchanged afterwards).
"""
import ctypes

import numpy as np
import pytest

from testmatrices import make_test_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def vp(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


@pytest.fixture
def torch_allocator(cuda_lib):
    cuda_lib.use_torch_allocator(True)
    yield cuda_lib
    cuda_lib.use_torch_allocator(False)


def test_factor_with_null_workspace(torch_allocator):
    P = torch_allocator
    L = P.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    A = P.colmajor(torch.from_numpy(make_test_matrix(30011, 64, 1e12, seed=6200)).cuda())
    Qw, Rw = P.factor(A, 16)
    Q, R = P.empty_colmajor(30011, 64, "cuda"), P.empty_colmajor(64, 64, "cuda")
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    rc = L.cqr_factor(30011, 64, vp(A), A.stride(1), 16, vp(Q), Q.stride(1), vp(R), R.stride(1), 0, None, 0, s)
    assert rc == 0
    assert torch.cuda.memory_allocated() == before
    assert torch.equal(Q, Qw) and torch.equal(R, Rw)
    # a breakdown comes back as the return value
    B = make_test_matrix(5000, 16, 1e3, seed=6201)
    B[:, 5] = 0.0
    Bt = P.colmajor(torch.from_numpy(B).cuda())
    Q2, R2 = P.empty_colmajor(5000, 16, "cuda"), P.empty_colmajor(16, 16, "cuda")
    rc = L.cqr_factor(5000, 16, vp(Bt), 5000, 4, vp(Q2), 5000, vp(R2), 16, 0, None, 0, s)
    assert rc == 6


def test_backward_and_batched_with_null_workspace(torch_allocator):
    P = torch_allocator
    L = P.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    m, n = 20000, 32
    A = P.colmajor(torch.from_numpy(make_test_matrix(m, n, 1e6, seed=6202)).cuda())
    Q, R = P.factor(A, 8)
    rng = np.random.default_rng(6203)
    dQ = P.colmajor(torch.from_numpy(rng.standard_normal((m, n))).cuda())
    dR = P.colmajor(torch.from_numpy(np.triu(rng.standard_normal((n, n)))).cuda())
    ref = P.backward(Q, R, dQ, dR)
    dA = P.empty_colmajor(m, n, "cuda")
    rc = L.cqr_backward(m, n, vp(Q), m, vp(R), n, vp(dQ), m, vp(dR), n, vp(dA), m, None, 0, s)
    assert rc == 0 and torch.equal(dA, ref)
    # batched
    As = [P.colmajor(torch.from_numpy(make_test_matrix(mm, nn, 1e5, seed=6204 + i)).cuda())
          for i, (mm, nn) in enumerate([(3000, 16), (9000, 32), (5000, 64)])]
    bs = [4, 8, 16]
    ref = P.factor_batched(As, bs)
    B = len(As)
    Qs = [P.empty_colmajor(a.shape[0], a.shape[1], "cuda") for a in As]
    Rs = [P.empty_colmajor(a.shape[1], a.shape[1], "cuda") for a in As]
    st = torch.full((B,), -7, dtype=torch.int32, device="cuda")
    i64 = ctypes.c_int64 * B
    rc = L.cqr_factor_batched(B, i64(*[a.shape[0] for a in As]), i64(*[a.shape[1] for a in As]),
                              i64(*[a.shape[0] for a in As]), (ctypes.c_int * B)(*bs),
                              (ctypes.c_void_p * B)(*[a.data_ptr() for a in As]),
                              (ctypes.c_void_p * B)(*[q.data_ptr() for q in Qs]),
                              (ctypes.c_void_p * B)(*[r.data_ptr() for r in Rs]), 0, vp(st), None, 0, s)
    assert rc == 0 and st.tolist() == [0, 0, 0]
    for (Qr, Rr), Qb, Rb in zip(ref, Qs, Rs):
        assert torch.equal(Qr, Qb) and torch.equal(Rr, Rb)
