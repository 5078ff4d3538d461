"""GPU adjoint of A = QR against the oracle, finite differences and torch.

Tolerance: the adjoint is a fixed sequence of products and one triangular
solve against R^T, so on the same (Q, R, Qbar, Rbar) the two sides differ by
rounding amplified by cond(R): ||dA_gpu - dA_oracle|| / ||dA_oracle|| <=
64 u cond(R) sqrt(n) (stated per test).
"""
import numpy as np
import pytest

from _helpers import U, rel_diff
from testmatrices import make_test_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(x):
    return torch.from_numpy(np.asfortranarray(x)).cuda()


@pytest.mark.parametrize("m,n,kappa", [(5000, 8, 10.0), (20000, 64, 1e4), (9001, 128, 1e3), (6000, 200, 1e2)])
def test_backward_matches_oracle(cuda_lib, oracle, m, n, kappa):
    P = cuda_lib
    A = make_test_matrix(m, n, kappa, seed=2000 + n)
    Q, R = oracle.mcqr2gs(A, n // 4 if n % 4 == 0 else n)
    rng = np.random.default_rng(2001)
    dQ = rng.standard_normal((m, n))
    dR = np.triu(rng.standard_normal((n, n)))
    dA_o = oracle.backward(Q, R, dQ, dR)
    dA_g = P.backward(_t(Q), _t(R), _t(dQ), _t(dR)).cpu().numpy()
    tol = 64 * U * np.linalg.cond(R) * np.sqrt(n)
    assert rel_diff(dA_g, dA_o) <= tol, (rel_diff(dA_g, dA_o), tol)


def test_backward_none_gradients(cuda_lib, oracle):
    P = cuda_lib
    A = make_test_matrix(3000, 16, 1e2, seed=2002)
    Q, R = oracle.mcqr2gs(A, 4)
    rng = np.random.default_rng(2003)
    dQ = rng.standard_normal((3000, 16))
    dR = np.triu(rng.standard_normal((16, 16)))
    g1 = P.backward(_t(Q), _t(R), _t(dQ), None).cpu().numpy()
    assert rel_diff(g1, oracle.backward(Q, R, dQ, np.zeros((16, 16)))) < 1e-12
    g2 = P.backward(_t(Q), _t(R), None, _t(dR)).cpu().numpy()
    assert rel_diff(g2, oracle.backward(Q, R, np.zeros((3000, 16)), dR)) < 1e-12


def test_autograd_finite_differences(cuda_lib):
    """Central differences of L = <Qbar, Q> + <Rbar, R> through the GPU
    forward, m = 500, n = 8 (all 4000 entries)."""
    P = cuda_lib
    m, n = 500, 8
    A = make_test_matrix(m, n, 1e2, seed=2004)
    rng = np.random.default_rng(2005)
    dQ = _t(rng.standard_normal((m, n)))
    dR = _t(np.triu(rng.standard_normal((n, n))))
    At = _t(A).requires_grad_(True)
    Q, R = P.qr(At, 4)
    ((Q * dQ).sum() + (R * dR).sum()).backward()
    g = At.grad.cpu().numpy()
    h = 1e-6
    Ab = _t(A)
    fd = np.zeros_like(A)
    # batch the perturbations column by column on the GPU
    for i in range(m):
        for j in range(n):
            Ap = Ab.clone()
            Ap[i, j] += h
            Am = Ab.clone()
            Am[i, j] -= h
            Qp, Rp = P.factor(P.colmajor(Ap), 4, check=False)
            Qm, Rm = P.factor(P.colmajor(Am), 4, check=False)
            fd[i, j] = float(((Qp - Qm) * dQ).sum() + ((Rp - Rm) * dR).sum()) / (2 * h)
    assert rel_diff(g, fd) < 1e-6


def test_autograd_matches_torch_linalg_qr(cuda_lib):
    P = cuda_lib
    m, n = 20000, 32
    A = make_test_matrix(m, n, 1e4, seed=2006)
    rng = np.random.default_rng(2007)
    dQ = _t(rng.standard_normal((m, n)))
    dR = _t(np.triu(rng.standard_normal((n, n))))
    At = _t(A).requires_grad_(True)
    Q, R = P.qr(At, 8)
    ((Q * dQ).sum() + (R * dR).sum()).backward()
    Bt = _t(A).contiguous().requires_grad_(True)
    Qt, Rt = torch.linalg.qr(Bt)
    D = torch.sign(torch.diagonal(Rt)).detach()
    ((Qt * D * dQ).sum() + (Rt * D[:, None] * dR).sum()).backward()
    assert rel_diff(At.grad.cpu().numpy(), Bt.grad.cpu().numpy()) < 1e-9
