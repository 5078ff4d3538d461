"""GPU (sm_103a) path against the CPU oracle, element by element.

Tolerances (FP64, u = 2^-53), from the accuracy targets of the library:
  * ||I - Q^T Q||_F <= 1e-13 and ||A - Q R||_F / ||A||_F <= 1e-14 for every
    kappa up to 1e15 (absolute targets, both sides must meet them);
  * R element-wise: ||R_gpu - R_oracle||_F / ||R_oracle||_F <= 1e-11 for
    kappa <= 1e6.  The two sides sum in different orders (split-m partials,
    fused multiply-adds), and R's forward error grows like kappa * u, so for
    larger kappa only the norms bind (parity unpinned there);
  * Q element-wise: max |Q_gpu - Q_oracle| <= 1e-11 for kappa <= 1e6;
  * exact dyadic inputs: bit-exact (every step is exact in IEEE arithmetic).
"""
import numpy as np
import pytest

from _helpers import exact_qr_case, load_exact_golden, orth_err, rel_diff, resid
from testmatrices import make_test_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORTH_TOL, RES_TOL, R_TOL, Q_TOL = 1e-13, 1e-14, 1e-11, 1e-11


def gpu_factor(P, A, b, variant, **kw):
    At = torch.from_numpy(np.asfortranarray(A)).cuda()
    At = P.colmajor(At)
    Q, R = P.factor(At, b, variant, **kw)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), R.cpu().numpy()


def oracle_factor(oracle, A, b, variant):
    return {
        "mcqr2gs": lambda: oracle.mcqr2gs(A, b),
        "cqr2gs": lambda: oracle.cqr2gs(A, b),
        "cqr2": lambda: oracle.cqr2(A),
        "scqr3": lambda: oracle.scqr3(A),
    }[variant]()


def check_against_oracle(P, oracle, A, b, variant, kappa, orth_tol=ORTH_TOL):
    Qg, Rg = gpu_factor(P, A, b, variant)
    Qo, Ro = oracle_factor(oracle, A, b, variant)
    assert np.all(np.tril(Rg, -1) == 0) and np.all(np.diag(Rg) > 0)
    assert orth_err(Qg) <= orth_tol, orth_err(Qg)
    assert resid(A, Qg, Rg) <= RES_TOL, resid(A, Qg, Rg)
    if kappa <= 1e6:
        assert rel_diff(Rg, Ro) <= R_TOL, rel_diff(Rg, Ro)
        assert np.abs(Qg - Qo).max() <= Q_TOL, np.abs(Qg - Qo).max()
    return Qg, Rg, Qo, Ro


# --------------------------------------------------------------------------- exact inputs: bit-exact
@pytest.mark.parametrize("variant", ["mcqr2gs", "cqr2gs", "cqr2"])
def test_exact_golden_bitwise(cuda_lib, variant):
    A, Q0, R0 = load_exact_golden()
    for b in (1, 2, 4, 8):
        Q, R = gpu_factor(cuda_lib, A, b, variant)
        assert np.array_equal(R, R0), (variant, b)
        assert np.array_equal(Q, Q0), (variant, b)


@pytest.mark.parametrize("m,n,b", [(4096, 64, 16), (16384, 128, 32), (4096, 96, 24), (1024, 12, 3)])
def test_exact_dyadic_bitwise(cuda_lib, oracle, m, n, b):
    A, Q0, R0 = exact_qr_case(m, n, seed=m + n)
    for variant in ("mcqr2gs", "cqr2gs"):
        Q, R = gpu_factor(cuda_lib, A, b, variant)
        assert np.array_equal(R, R0) and np.array_equal(Q, Q0), variant


# --------------------------------------------------------------------------- against the oracle
@pytest.mark.parametrize("variant", ["mcqr2gs", "cqr2gs"])
@pytest.mark.parametrize("m,n,b,kappa", [
    (20000, 64, 16, 1e10),     # the 20,000 x 64, b = 16 workload
    (20000, 64, 16, 1e4),
    (30011, 48, 16, 1e6),      # ragged m: not a multiple of any tile or row block
    (9999, 40, 8, 1e5),
    (5000, 30, 10, 1e3),       # widths that are not multiples of 4 or 8
    (4097, 9, 3, 1e2),
    (3000, 7, 1, 1e2),         # b = 1
    (12000, 128, 64, 1e6),
    (8000, 256, 128, 1e6),     # the widest one-block Cholesky / TRSM
    (6000, 256, 256, 1e3),     # blocked Gram, Cholesky in L2, blocked TRSM
])
def test_parity(cuda_lib, oracle, variant, m, n, b, kappa):
    A = make_test_matrix(m, n, kappa, seed=1000 + m + n + b)
    check_against_oracle(cuda_lib, oracle, A, b, variant, kappa)


@pytest.mark.parametrize("kappa", [1e2, 1e5, 1e8, 1e12, 1e15])
def test_parity_kappa_sweep_mcqr2gs(cuda_lib, oracle, kappa):
    A = make_test_matrix(20000, 60, kappa, seed=1100)
    check_against_oracle(cuda_lib, oracle, A, 20, "mcqr2gs", kappa)


def test_parity_cqr2gs_ten_panels_at_1e15(cuda_lib, oracle):
    A = make_test_matrix(20000, 60, 1e15, seed=1101)
    check_against_oracle(cuda_lib, oracle, A, 6, "cqr2gs", 1e15)


@pytest.mark.parametrize("m,n", [(20000, 64), (7001, 160), (3000, 1)])
def test_parity_cqr2(cuda_lib, oracle, m, n):
    A = make_test_matrix(m, n, 1e5, seed=1200 + n)
    check_against_oracle(cuda_lib, oracle, A, n, "cqr2", 1e5)


@pytest.mark.parametrize("kappa", [1e3, 1e6, 1e12])
def test_parity_scqr3(cuda_lib, oracle, kappa):
    """Shifted CholeskyQR3 (Alg. 5): the shift s = sqrt(m) u ||A||_F^2 (Alg. 4)
    acts at every kappa, so the element-wise comparison at kappa <= 1e6 binds
    the shifted first pass; at 1e12 only the norms bind."""
    A = make_test_matrix(20000, 48, kappa, seed=1300)
    check_against_oracle(cuda_lib, oracle, A, 48, "scqr3", kappa)


def test_square_and_single_column(cuda_lib, oracle):
    A = make_test_matrix(64, 64, 1e3, seed=1400)
    check_against_oracle(cuda_lib, oracle, A, 16, "mcqr2gs", 1e3)
    A = make_test_matrix(100, 1, 1.0, seed=1401)
    check_against_oracle(cuda_lib, oracle, A, 1, "mcqr2gs", 1.0)


# --------------------------------------------------------------------------- layouts, aliasing, determinism
def test_inplace_and_padded_lda(cuda_lib):
    P = cuda_lib
    A = make_test_matrix(10000, 32, 1e6, seed=1500)
    Q1, R1 = gpu_factor(P, A, 8, "mcqr2gs")
    buf = torch.zeros((32, 10240), dtype=torch.float64, device="cuda")
    Ap = buf.t()[:10000]  # lda = 10240
    Ap.copy_(torch.from_numpy(A))
    Q2, R2 = P.factor(Ap, 8, "mcqr2gs", inplace=True)
    assert Q2.data_ptr() == Ap.data_ptr()
    assert np.array_equal(Q2.cpu().numpy(), Q1) and np.array_equal(R2.cpu().numpy(), R1)
    assert float(buf.t()[10000:].abs().max()) == 0.0  # padding rows untouched


def test_deterministic(cuda_lib):
    A = make_test_matrix(50000, 64, 1e8, seed=1501)
    Q1, R1 = gpu_factor(cuda_lib, A, 16, "mcqr2gs")
    Q2, R2 = gpu_factor(cuda_lib, A, 16, "mcqr2gs")
    assert np.array_equal(Q1, Q2) and np.array_equal(R1, R2)


@pytest.mark.parametrize("variant,b", [("mcqr2gs", 16), ("cqr2gs", 8)])
def test_lookahead_is_bitwise_identical(cuda_lib, variant, b):
    """Look-ahead (Sec. 7 future work) only reorders launches across two
    streams; every element sees the same FMA sequence."""
    A = make_test_matrix(50000, 96, 1e12, seed=1503)
    Q1, R1 = gpu_factor(cuda_lib, A, b, variant)
    Q2, R2 = gpu_factor(cuda_lib, A, b, variant, lookahead=True)
    assert np.array_equal(Q1, Q2) and np.array_equal(R1, R2)


@pytest.mark.parametrize("variant,b,kappa", [("mcqr2gs", 16, 1e5), ("cqr2gs", 8, 1e5), ("mcqr2gs", 24, 1e15)])
def test_lookahead_against_oracle(cuda_lib, oracle, variant, b, kappa):
    """The look-ahead schedule against the oracle's plain Alg. 9 / Alg. 7
    (not only against the GPU's default schedule): element-wise at 1e5,
    norms at 1e15."""
    A = make_test_matrix(40001, 96, kappa, seed=1505)
    Qg, Rg = gpu_factor(cuda_lib, A, b, variant, lookahead=True)
    Qo, Ro = oracle_factor(oracle, A, b, variant)
    assert np.all(np.tril(Rg, -1) == 0) and np.all(np.diag(Rg) > 0)
    assert orth_err(Qg) <= ORTH_TOL and resid(A, Qg, Rg) <= RES_TOL
    if kappa <= 1e6:
        assert rel_diff(Rg, Ro) <= R_TOL and np.abs(Qg - Qo).max() <= Q_TOL


@pytest.mark.parametrize("kappa", [1.0, 1e10])
def test_adaptive_repetitions_match_oracle(cuda_lib, oracle, kappa):
    """Runtime choice of the second CholeskyQR pass (Sec. 7): at kappa = 1 the
    rule fires on every panel (both sides), at 1e10 never; parity with the
    oracle's adaptive mode either way."""
    A = make_test_matrix(30000, 64, kappa, seed=1504)
    Qg, Rg = gpu_factor(cuda_lib, A, 16, "mcqr2gs", adaptive=True)
    Qo, Ro = oracle.mcqr2gs(A, 16, adaptive=True)
    assert orth_err(Qg) <= ORTH_TOL and resid(A, Qg, Rg) <= RES_TOL
    if kappa <= 1e6:
        assert rel_diff(Rg, Ro) <= R_TOL and np.abs(Qg - Qo).max() <= Q_TOL
    if kappa == 1.0:  # skipped passes: R_jj = S1 exactly, so S2 = I on both sides
        Qd, Rd = gpu_factor(cuda_lib, A, 16, "mcqr2gs")
        assert not np.array_equal(Qd, Qg)
    else:
        Qd, Rd = gpu_factor(cuda_lib, A, 16, "mcqr2gs")
        assert np.array_equal(Qd, Qg) and np.array_equal(Rd, Rg)


def test_side_stream(cuda_lib):
    A = make_test_matrix(20000, 32, 1e4, seed=1502)
    Q1, R1 = gpu_factor(cuda_lib, A, 8, "mcqr2gs")
    s = torch.cuda.Stream()
    At = cuda_lib.colmajor(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        Q2, R2 = cuda_lib.factor(At, 8, "mcqr2gs", stream=s)
    s.synchronize()
    assert np.array_equal(Q2.cpu().numpy(), Q1) and np.array_equal(R2.cpu().numpy(), R1)


# --------------------------------------------------------------------------- failures and arguments
def test_breakdown_status_and_recovery(cuda_lib, oracle):
    """An exactly zero column makes the radicand exactly 0 (Sec. 3: the Gram
    matrix is not positive definite): both sides report the same column;
    a NaN input is a breakdown too; the context stays usable."""
    P = cuda_lib
    A = make_test_matrix(5000, 16, 1e3, seed=1600)
    A[:, 5] = 0.0
    _, _, st_o = oracle.mcqr2gs(A, 4, check=False)
    with pytest.raises(P.CQRError) as ei:
        gpu_factor(P, A, 4, "mcqr2gs")
    assert ei.value.code == st_o == 6
    An = make_test_matrix(5000, 16, 1e3, seed=1600)
    An[17, 3] = np.nan
    with pytest.raises(P.CQRError) as ei:
        gpu_factor(P, An, 4, "mcqr2gs")
    assert ei.value.code > 0
    B = make_test_matrix(5000, 16, 1e3, seed=1601)
    Q, R = gpu_factor(P, B, 4, "mcqr2gs")
    assert orth_err(Q) < ORTH_TOL


def test_breakdown_column_matches_oracle(cuda_lib, oracle):
    A = make_test_matrix(4000, 12, 1e2, seed=1602)
    A[:, 9] = 0.0  # exactly zero column: the radicand is exactly 0 at column 9
    _, _, st_o = oracle.cqr2(A, check=False)
    with pytest.raises(cuda_lib.CQRError) as ei:
        gpu_factor(cuda_lib, A, 12, "cqr2")
    assert ei.value.code == st_o == 10


def test_argument_errors(cuda_lib):
    import ctypes

    P = cuda_lib
    L = P.load()
    A = torch.zeros((16, 100), dtype=torch.float64, device="cuda").t()
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    R = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.cqr_factor(10, 16, p(A), 100, 4, p(A), 100, p(R), 16, 0, p(ws), ws.numel(), s) == -1  # m < n
    assert L.cqr_factor(100, 16, p(A), 50, 4, p(A), 50, p(R), 16, 0, p(ws), ws.numel(), s) == -4  # lda < m
    assert L.cqr_factor(100, 16, p(A), 100, 5, p(A), 100, p(R), 16, 0, p(ws), ws.numel(), s) == -5  # b !| n
    assert L.cqr_factor(100, 16, p(A), 100, 4, p(A), 100, p(R), 8, 0, p(ws), ws.numel(), s) == -9  # ldr < n
    assert L.cqr_factor(100, 16, p(A), 100, 4, p(A), 100, p(R), 16, 7, p(ws), ws.numel(), s) == -10
    assert L.cqr_factor(100, 16, p(A), 100, 4, p(A), 100, p(R), 16, 0, p(ws), 16, s) == -12  # small ws
    assert L.cqr_factor(100, 16, p(A), 100, 4, p(A), 100, p(R), 16, 0, ctypes.c_void_p(ws.data_ptr() + 8),
                        ws.numel() - 8, s) == -11  # misaligned ws
    torch.cuda.synchronize()
