"""Emulated products (CQR_EMULATED): the m-row products of Alg. 9 (Gram
matrices, projections Y = Q^T A and Z = Q^T P, updates A -= Q Y and
P -= Q Z) on the tcgen05 FP8 tensor cores with the error-free (Ozaki)
splitting, checked against the FP64 oracle with the tolerances of the native
path (orthogonality <= 1e-13, residual <= 1e-14, R <= 1e-11 for kappa <= 1e6)
and bit for bit on exact dyadic inputs, where every digit product and every
sum is exact."""
import numpy as np
import pytest

from _helpers import exact_qr_case, load_exact_golden, orth_err, rel_diff, resid
from testmatrices import make_test_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu_factor(P, A, b, **kw):
    At = P.colmajor(torch.from_numpy(np.asfortranarray(A)).cuda())
    Q, R = P.factor(At, b, "mcqr2gs", **kw)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), R.cpu().numpy()


def test_emulated_exact_golden(cuda_lib):
    A, Q0, R0 = load_exact_golden()
    for b in (1, 2, 4, 8):
        Q, R = gpu_factor(cuda_lib, A, b, emulated=True)
        assert np.array_equal(R, R0) and np.array_equal(Q, Q0), b


@pytest.mark.parametrize("m,n,b", [(4096, 64, 16), (16384, 128, 32), (1024, 12, 3),
                                   (4096, 96, 48)])  # b = 48: a 16-column substitution block after a 32-column one
def test_emulated_exact_dyadic(cuda_lib, m, n, b):
    A, Q0, R0 = exact_qr_case(m, n, seed=m + n)
    Q, R = gpu_factor(cuda_lib, A, b, emulated=True)
    assert np.array_equal(R, R0) and np.array_equal(Q, Q0)


@pytest.mark.parametrize("m,n,b,kappa", [
    (20000, 64, 16, 1e10),
    (30011, 48, 16, 1e6),     # ragged m: partial last sub-chunk
    (9999, 40, 8, 1e5),
    (12000, 128, 32, 1e4),
    (50000, 256, 64, 1e15),
    (8000, 96, 24, 1e12),
    (8192, 1536, 128, 1e5),   # re-orthogonalisation updates with K = jb > 1312: the F2I level-sum path
    (30011, 96, 48, 1e6),     # ragged m; the solve's coupling product has N = 16 (a partial column tile)
])
def test_emulated_parity(cuda_lib, oracle, m, n, b, kappa):
    A = make_test_matrix(m, n, kappa, seed=5000 + m + n)
    Qg, Rg = gpu_factor(cuda_lib, A, b, emulated=True)
    Qo, Ro = oracle.mcqr2gs(A, b)
    assert np.all(np.tril(Rg, -1) == 0) and np.all(np.diag(Rg) > 0)
    assert orth_err(Qg) <= 1e-13, orth_err(Qg)
    assert resid(A, Qg, Rg) <= 1e-14, resid(A, Qg, Rg)
    if kappa <= 1e6:
        assert rel_diff(Rg, Ro) <= 1e-11, rel_diff(Rg, Ro)
        assert np.abs(Qg - Qo).max() <= 1e-11


def test_emulated_zero_and_nan_columns(cuda_lib, oracle):
    """A zero column gives an exactly zero scale (status = breakdown column
    like the native path); a NaN reaches the Cholesky as a breakdown."""
    P = cuda_lib
    A = make_test_matrix(9000, 32, 1e3, seed=5100)
    A[:, 13] = 0.0
    with pytest.raises(P.CQRError) as ei:
        gpu_factor(P, A, 8, emulated=True)
    _, _, st = oracle.mcqr2gs(A, 8, check=False)
    assert ei.value.code == st == 14
    A = make_test_matrix(9000, 32, 1e3, seed=5101)
    A[4444, 20] = np.nan
    with pytest.raises(P.CQRError) as ei:
        gpu_factor(P, A, 8, emulated=True)
    assert ei.value.code > 0


def test_emulated_contraction_beyond_one_chunk(cuda_lib):
    """n > 4096 + b: the re-orthogonalisation update contracts over more than
    4096 columns, so it runs in several contraction chunks (each with exact
    level sums), and the Z projection spans 34 row tiles.  Checked against
    the native FP64 factorisation on the GPU (kappa = 1e5, R within 1e-11)
    and by the norms."""
    P = cuda_lib
    m, n, b = 8192, 4352, 64
    A = P.colmajor(torch.from_numpy(make_test_matrix(m, n, 1e5, seed=5200)).cuda())
    Qe, Re = P.factor(A, b, "mcqr2gs", emulated=True)
    Qn, Rn = P.factor(A, b, "mcqr2gs")
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    assert torch.linalg.norm(eye - Qe.t() @ Qe).item() <= 1e-13 * (n / 1024)
    assert (torch.linalg.norm(A - Qe @ Re) / torch.linalg.norm(A)).item() <= 1e-14
    assert (torch.linalg.norm(Re - Rn) / torch.linalg.norm(Rn)).item() <= 1e-11
