"""Pins of the CPU oracle against things other than itself (no GPU).

Each test fixes the oracle with an independent fact:
  * the exact QR of a dyadic input (closed form, tests/golden),
  * Householder QR by brute force on tiny inputs (LAPACK via numpy, and the
    oracle's own textbook Householder, itself pinned to LAPACK),
  * closed forms: R_11 = ||a_1||, orthogonal columns give a diagonal R,
  * reductions stated by the paper: b = n turns CQR2GS into CQR2 (Sec. 5.3)
    and Alg. 9 with one panel is CQR2 (its step 1),
  * the paper's stability claims (Sec. 4, 5.3, 5.4) on scaled-down matrices,
  * a planted mistake (the paper-literal R of Alg. 9, which omits the
    re-orthogonalisation coefficients) must be caught by the residual pin,
  * finite differences and torch.linalg.qr for the adjoint,
  * the adaptive panel width (or_mcqr2gs_halving) against the pinned
    or_mcqr2gs: identical when no panel is rejected, identical to the
    narrower width when the first panel is, decisions equal to the rule
    evaluated independently (LAPACK Cholesky of numpy's Gram matrix), and
    the paper's O(u) accuracy where plain two-panel mCQR2GS breaks down.
"""
import numpy as np
import pytest

from _helpers import U, exact_qr_case, load_exact_golden, orth_err, rel_diff, resid, sign_normalised_qr
from testmatrices import gaussian, make_test_matrix, sigma

VARIANTS = ["mcqr2gs", "cqr2gs", "cqr2"]


def run(oracle, variant, A, b, check=True):
    if variant == "mcqr2gs":
        return oracle.mcqr2gs(A, b, check=check)
    if variant == "cqr2gs":
        return oracle.cqr2gs(A, b, check=check)
    if variant == "cqr2":
        return oracle.cqr2(A, check=check)
    if variant == "scqr3":
        return oracle.scqr3(A, check=check)
    raise ValueError(variant)


# --------------------------------------------------------------------------- exact golden
@pytest.mark.parametrize("variant", VARIANTS + ["scqr3_gram"])
def test_exact_golden_fixture(oracle, variant):
    A, Q0, R0 = load_exact_golden()
    if variant == "scqr3_gram":
        # the Gram step alone: W = A^T A = R0^T R0 exactly (integers)
        W = oracle.gram(A)
        assert np.array_equal(W, R0.T @ R0)
        U_, st = oracle.chol(W)
        assert st == 0 and np.array_equal(U_, R0)
        return
    for b in (1, 2, 4, 8):
        Q, R = run(oracle, variant, A, b)
        assert np.array_equal(R, R0), (variant, b)
        assert np.array_equal(Q, Q0), (variant, b)


@pytest.mark.parametrize("seed", range(3))
def test_exact_dyadic_cases(oracle, seed):
    A, Q0, R0 = exact_qr_case(256, 16, seed)
    for variant in VARIANTS:
        for b in (4, 8, 16):
            Q, R = run(oracle, variant, A, b)
            assert np.array_equal(R, R0) and np.array_equal(Q, Q0), (variant, b)


# --------------------------------------------------------------------------- brute force vs Householder
def test_householder_matches_lapack(oracle):
    rng = np.random.default_rng(7)
    for m, n in [(1, 1), (5, 1), (7, 3), (20, 8), (64, 8), (40, 40)]:
        A = rng.standard_normal((m, n))
        Q, R = oracle.householder(A)
        Qn, Rn = sign_normalised_qr(A)
        assert np.allclose(R, Rn, rtol=0, atol=1e-13 * np.abs(Rn).max())
        assert np.allclose(Q, Qn, rtol=0, atol=1e-13)
        assert np.all(np.diag(R) >= 0) and np.allclose(np.tril(R, -1), 0)


@pytest.mark.parametrize("m", [8, 13, 33, 64])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("kappa", [1.0, 1e3, 1e6])
def test_brute_force_vs_householder(oracle, m, n, kappa):
    if n > m:
        pytest.skip("m >= n")
    A = make_test_matrix(m, n, kappa, seed=100 + m * 10 + n)
    Qh, Rh = oracle.householder(A)
    tol = 50 * max(kappa, 1.0) * U * max(n, 2)
    for variant in VARIANTS:
        for b in [d for d in range(1, n + 1) if n % d == 0]:
            Q, R = run(oracle, variant, A, b)
            assert rel_diff(R, Rh) < tol, (variant, b, rel_diff(R, Rh))
            assert np.abs(Q - Qh).max() < tol, (variant, b)
            assert np.allclose(np.tril(R, -1), 0.0, atol=0) and np.all(np.diag(R) > 0)


# --------------------------------------------------------------------------- closed forms
def test_r11_is_column_norm(oracle):
    A = gaussian(500, 6, seed=3)
    for variant in VARIANTS:
        _, R = run(oracle, variant, A, 2)
        assert abs(R[0, 0] - np.linalg.norm(A[:, 0])) < 4 * U * R[0, 0]


def test_orthogonal_columns_give_diagonal_r(oracle):
    A, Q0, _ = exact_qr_case(256, 12, seed=11)
    d = np.array([3.0, 0.5, 7.0, 1.0, 2.0, 11.0, 0.25, 5.0, 9.0, 1.5, 4.0, 6.0])
    Ad = Q0 * d
    for variant in VARIANTS:
        for b in (3, 4, 6, 12):
            Q, R = run(oracle, variant, Ad, b)
            assert np.allclose(R, np.diag(d), rtol=0, atol=8 * U * d.max())
            assert orth_err(Q) < 1e-14


def test_gram_and_tn_definitions(oracle):
    X = gaussian(1000, 5, seed=4)
    Y = gaussian(1000, 3, seed=5)
    W = oracle.gram(X)
    assert np.array_equal(W, W.T)
    assert np.allclose(W, X.T @ X, rtol=1e-14, atol=0)
    T = oracle.tn(X, Y)
    assert np.allclose(T, X.T @ Y, rtol=0, atol=1e-12)
    Z = oracle.update(Y, X, np.ones((5, 3)))
    assert np.allclose(Z, Y - X @ np.ones((5, 3)), rtol=0, atol=1e-12)


def test_chol_definition_and_breakdown(oracle):
    rng = np.random.default_rng(1)
    B = rng.standard_normal((30, 6))
    W = B.T @ B
    Uc, st = oracle.chol(W)
    assert st == 0
    L = np.linalg.cholesky(W)  # LAPACK, lower
    assert np.allclose(Uc, L.T, rtol=0, atol=1e-12 * np.abs(L).max())
    # not positive definite at column 3 (0-based 2): status = 3
    W2 = np.diag([4.0, 1.0, -1.0, 2.0])
    _, st = oracle.chol(W2)
    assert st == 3
    W3 = np.diag([1.0, np.nan, 1.0])
    _, st = oracle.chol(W3)
    assert st == 2


def test_trsm_is_right_solve(oracle):
    rng = np.random.default_rng(2)
    Ut = np.triu(rng.standard_normal((7, 7))) + 4 * np.eye(7)
    X = rng.standard_normal((50, 7))
    Q = oracle.trsm(X, Ut)
    assert np.allclose(Q @ Ut, X, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------- the paper's reductions
@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_b_equals_n_reduces_to_cqr2(oracle, kappa):
    """Sec. 5.3: b = n makes CQR2GS fall back to CholeskyQR2; Alg. 9 step 1
    makes one-panel mCQR2GS CholeskyQR2.  Same operation sequence: bitwise."""
    A = make_test_matrix(2000, 16, kappa, seed=21)
    Qc, Rc = oracle.cqr2(A)
    for variant in ("mcqr2gs", "cqr2gs"):
        Q, R = run(oracle, variant, A, 16)
        assert np.array_equal(Q, Qc) and np.array_equal(R, Rc)


def test_block_rows_floor(oracle):
    """Two valid summation orders differ by a rounding-level amount: the
    achievable parity floor for a different (GPU) order."""
    A = make_test_matrix(30000, 32, 1e6, seed=22)
    Q1, R1 = oracle.mcqr2gs(A, 8)
    try:
        oracle.set_block_rows(1)
        Q2, R2 = oracle.mcqr2gs(A, 8)
    finally:
        oracle.set_block_rows(4096)
    d = rel_diff(R2, R1)
    assert 0 < d < 1e-11, d


# --------------------------------------------------------------------------- invariants at moderate size
@pytest.mark.parametrize("variant,b", [("mcqr2gs", 16), ("cqr2gs", 16), ("cqr2", 64)])
def test_invariants(oracle, variant, b):
    A = make_test_matrix(20000, 64, 1e4, seed=23)
    Q, R = run(oracle, variant, A, b)
    assert np.allclose(np.tril(R, -1), 0, atol=0) and np.all(np.diag(R) > 0)
    assert orth_err(Q) < 1e-13 and resid(A, Q, R) < 1e-14
    assert rel_diff(R.T @ R, A.T @ A) < 1e-14 * 1e4
    # Q spans A: (I - Q Q^T) A small
    P = A - Q @ (Q.T @ A)
    assert np.linalg.norm(P) / np.linalg.norm(A) < 1e-14


# --------------------------------------------------------------------------- the paper's stability claims
def test_cqr2_unstable_beyond_1e8(oracle):
    """Sec. 4: CholeskyQR2 is stable only up to kappa ~ u^{-1/2} ~ 1e8."""
    A = make_test_matrix(3000, 60, 1e6, seed=31)
    Q, R = oracle.cqr2(A)
    assert orth_err(Q) < 1e-13
    A = make_test_matrix(3000, 60, 1e15, seed=31)
    Q, R, st = oracle.cqr2(A, check=False)
    assert st != 0 or orth_err(Q) > 1e-6


def test_mcqr2gs_three_panels_at_1e15(oracle):
    """Sec. 5.4, Fig. 6: at kappa = 1e15 mCQR2GS with 3 panels reaches O(u)
    orthogonality and residual."""
    A = make_test_matrix(6000, 600, 1e15, seed=32)
    Q3, R3 = oracle.mcqr2gs(A, 200)
    assert orth_err(Q3) < 1e-13 and resid(A, Q3, R3) < 1e-14


def test_two_panel_first_panel_at_breakdown_edge():
    """Sec. 5.4: with 2 panels at kappa = 1e15 the first panel's condition is
    bounded below by about 1e8 (Eq. cond_bounds), so its Gram matrix reaches
    cond ~ u^{-1}: CholeskyQR on it is at the edge of breakdown.  With 3
    panels the first panel is far better conditioned."""
    A = make_test_matrix(6000, 600, 1e15, seed=32)
    c2 = np.linalg.cond(A[:, :300])
    c3 = np.linalg.cond(A[:, :200])
    assert c2 > 3e7 and c2 ** 2 > 0.5e15
    assert c3 < 1e7


def test_panel_condition_interlacing_bounds():
    """Sec. 5.3, Eq. cond_bounds: for B = the first r columns of A,
    cond(A) >= cond(B) >= sigma_{1+(n-r)} / sigma_r."""
    A = make_test_matrix(2000, 40, 1e12, seed=36)
    s = np.linalg.svd(A, compute_uv=False)
    n = 40
    for r in (5, 10, 20, 30):
        cb = np.linalg.cond(A[:, :r])
        assert s[0] / s[-1] * (1 + 1e-6) >= cb >= s[n - r] / s[r - 1] * (1 - 1e-6)


def test_cqr2gs_needs_ten_panels_at_1e15(oracle):
    """Sec. 5.3, Fig. 3: at kappa = 1e15 CQR2GS needs about 10 panels for
    O(u) orthogonality; with 2 panels orthogonality is lost, while mCQR2GS
    (Alg. 9) is already at O(u) with the same 2-3 panels (Sec. 5.4)."""
    A = make_test_matrix(6000, 600, 1e15, seed=34)
    Q, R, st = oracle.cqr2gs(A, 300, check=False)
    assert st != 0 or orth_err(Q) > 1e-6
    Q, R = oracle.cqr2gs(A, 60)
    assert orth_err(Q) < 1e-13 and resid(A, Q, R) < 1e-14
    Qm, Rm = oracle.mcqr2gs(A, 200)
    assert orth_err(Qm) < 1e-13


def test_scqr3_survives_1e15(oracle):
    """Sec. 5.2, Fig. 1: shifted CholeskyQR3 completes at kappa up to 1e15."""
    A = make_test_matrix(3000, 30, 1e12, seed=35)
    Q, R = oracle.scqr3(A)
    assert orth_err(Q) < 1e-13 and resid(A, Q, R) < 1e-14


def test_scqr_shift_closed_form(oracle):
    """Alg. 4 on exactly orthonormal columns (scaled Hadamard, every Gram sum
    exact): W = I, the shift is s = sqrt(m) u ||A||_F^2 = sqrt(m) u n, so the
    shifted Cholesky factor is sqrt(1 + s) I and Q = A / sqrt(1 + s), bit for
    bit.  A wrong sign of the shift, a missing sqrt(m) or a shift off the
    diagonal each changes the result."""
    for m, n in [(4096, 16), (1024, 12), (256, 3)]:
        _, Q0, _ = exact_qr_case(m, n, seed=m + n)
        s = np.sqrt(float(m)) * U * n
        assert s > 0 and (1.0 + s) != 1.0
        d = np.sqrt(1.0 + s)
        Q1, R1 = oracle.scqr(Q0)
        assert np.array_equal(R1, d * np.eye(n)), (m, n)
        assert np.array_equal(Q1, Q0 / d), (m, n)


def test_literal_r_reading_is_rounding_level(oracle):
    """Alg. 9 leaves R of steps 6-8 implicit.  Adding the re-orthogonalisation
    coefficients (R_{1:j-1,j} += Z S1) is exact in exact arithmetic; dropping
    them (the paper-literal R_jj = S2 S1 only) leaves a residual that is still
    O(u) but measurably larger, because Z is itself a rounding-level
    quantity once the projection of steps 3-4 has been applied."""
    A = make_test_matrix(3000, 60, 1e15, seed=32)
    Q, R = oracle.mcqr2gs(A, 20)
    Ql, Rl = oracle.mcqr2gs(A, 20, literal_r=True)
    assert np.array_equal(Q, Ql)
    assert resid(A, Q, R) < 1e-15
    assert 2 * resid(A, Q, R) < resid(A, Ql, Rl) < 1e-13


# --------------------------------------------------------------------------- runtime CQR repetition choice
@pytest.mark.parametrize("kappa", [1e4, 1e15])
def test_adaptive_rule_silent_on_ill_conditioned_panels(oracle, kappa):
    """Sec. 7 (runtime choice of the number of CholeskyQR repetitions): the
    second pass is skipped only when its factor is within 8u of I.  Panels of
    the paper's test matrices with kappa >= 1e2 never qualify, so the result
    is bitwise the default one."""
    A = make_test_matrix(20000, 64, kappa, seed=51)
    Q, R = oracle.mcqr2gs(A, 16)
    Qa, Ra = oracle.mcqr2gs(A, 16, adaptive=True)
    assert np.array_equal(Q, Qa) and np.array_equal(R, Ra)


def test_adaptive_rule_fires_on_orthonormal_panels(oracle):
    """kappa = 1: after the first pass every panel is orthonormal to working
    precision, the second pass is skipped, and the result stays O(u)."""
    A = make_test_matrix(20000, 64, 1.0, seed=52)
    Q, R = oracle.mcqr2gs(A, 16)
    Qa, Ra = oracle.mcqr2gs(A, 16, adaptive=True)
    assert not np.array_equal(Q, Qa)  # the rule did change the computation
    assert orth_err(Qa) < 1e-14 and resid(A, Qa, Ra) < 1e-15
    assert np.abs(Qa - Q).max() < 1e-15 and rel_diff(Ra, R) < 1e-15


# --------------------------------------------------------------------------- adjoint
def _loss_grad_fd(oracle, A, dQ, dR, b, h):
    G = np.zeros_like(A)
    for i in range(A.shape[0]):
        for j in range(A.shape[1]):
            Ap = A.copy(order="F")
            Am = A.copy(order="F")
            Ap[i, j] += h
            Am[i, j] -= h
            Qp, Rp = oracle.mcqr2gs(Ap, b)
            Qm, Rm = oracle.mcqr2gs(Am, b)
            lp = np.sum(dQ * Qp) + np.sum(dR * Rp)
            lm = np.sum(dQ * Qm) + np.sum(dR * Rm)
            G[i, j] = (lp - lm) / (2 * h)
    return G


@pytest.mark.parametrize("kappa", [10.0, 1e4])
def test_backward_finite_differences(oracle, kappa):
    m, n = 60, 8
    A = make_test_matrix(m, n, kappa, seed=41)
    rng = np.random.default_rng(42)
    dQ = rng.standard_normal((m, n))
    dR = np.triu(rng.standard_normal((n, n)))
    Q, R = oracle.mcqr2gs(A, 4)
    G = oracle.backward(Q, R, dQ, dR)
    h = 1e-6 * np.linalg.norm(A) / np.sqrt(m * n)
    Gfd = _loss_grad_fd(oracle, A, dQ, dR, 4, h)
    assert rel_diff(G, Gfd) < 1e-6 * max(1.0, kappa / 1e2)


def test_backward_matches_torch_autograd(oracle):
    torch = pytest.importorskip("torch")
    m, n = 200, 12
    A = make_test_matrix(m, n, 1e3, seed=43)
    rng = np.random.default_rng(44)
    dQ = rng.standard_normal((m, n))
    dR = np.triu(rng.standard_normal((n, n)))
    At = torch.tensor(A, requires_grad=True)
    Qt, Rt = torch.linalg.qr(At)
    D = torch.sign(torch.diagonal(Rt)).detach()
    Qs, Rs = Qt * D, Rt * D[:, None]
    loss = (Qs * torch.tensor(dQ)).sum() + (Rs * torch.tensor(dR)).sum()
    loss.backward()
    Q, R = oracle.mcqr2gs(A, 4)
    G = oracle.backward(Q, R, dQ, dR)
    assert rel_diff(G, At.grad.numpy()) < 1e-10


def test_backward_ignores_lower_rbar(oracle):
    A = make_test_matrix(100, 6, 1e2, seed=45)
    Q, R = oracle.cqr2(A)
    rng = np.random.default_rng(46)
    dQ = rng.standard_normal((100, 6))
    dR = rng.standard_normal((6, 6))
    G1 = oracle.backward(Q, R, dQ, dR)
    G2 = oracle.backward(Q, R, dQ, np.triu(dR))
    assert rel_diff(G1, G2) < 1e-14


def test_sigma_recipe():
    s = sigma(5, 1e8)
    assert s[0] == 1.0 and abs(s[-1] - 1e-8) < 1e-22 and np.all(np.diff(s) < 0)
    A = make_test_matrix(300, 10, 1e6, seed=1)
    sv = np.linalg.svd(A, compute_uv=False)
    assert abs(sv[0] / sv[-1] / 1e6 - 1) < 1e-6


# --------------------------------------------------------------------------- adaptive panel width
U_RULE = 1.0 / (64.0 * 2.0 ** -53)  # panel rejected when (max U_ii / min U_ii)^2 exceeds this


def independent_reject(X):
    """The panel test evaluated outside the oracle: LAPACK Cholesky of numpy's
    Gram matrix; a breakdown (not positive definite) rejects too."""
    try:
        L = np.linalg.cholesky(X.T @ X)
    except np.linalg.LinAlgError:
        return True
    d = np.diag(L)
    return (d.max() / d.min()) ** 2 > U_RULE


@pytest.mark.parametrize("m,n,b,kappa,seed", [(2000, 40, 20, 1e3, 21), (3000, 60, 20, 1e6, 22),
                                               (2000, 40, 20, 1e15, 1), (4000, 80, 40, 1e15, 2)])
def test_halving_without_rejection_is_mcqr2gs(oracle, m, n, b, kappa, seed):
    """No panel rejected: exactly Alg. 9 with the given width."""
    A = make_test_matrix(m, n, kappa, seed)
    assert not independent_reject(A[:, :b])
    Q, R, bf = oracle.mcqr2gs_halving(A, b)
    Q0, R0 = oracle.mcqr2gs(A, b)
    assert bf == b and np.array_equal(Q, Q0) and np.array_equal(R, R0)


@pytest.mark.parametrize("seed,why", [(3, "breakdown"), (8, "ratio")])
def test_halving_at_the_first_panel_is_the_narrower_width(oracle, seed, why):
    """The first panel rejected (seed 3: its Cholesky breaks down; seed 8: no
    breakdown, but the diagonal ratio is ~10x over the bound) and nothing
    later: exactly Alg. 9 with b = 10 from the start."""
    A = make_test_matrix(2000, 40, 1e15, seed)
    _, st = oracle.chol(oracle.gram(A[:, :20]))
    assert (st != 0) == (why == "breakdown")
    if why == "ratio":  # far from the bound: the same decision outside the oracle
        assert independent_reject(A[:, :20])
    Q, R, bf = oracle.mcqr2gs_halving(A, 20)
    Q0, R0 = oracle.mcqr2gs(A, 10)
    assert bf == 10 and np.array_equal(Q, Q0) and np.array_equal(R, R0)


@pytest.mark.parametrize("m,n,seed", [(2000, 40, 2), (2000, 40, 6), (4000, 80, 6), (4000, 80, 9), (6000, 120, 2)])
def test_halving_recovers_where_two_panels_break_down(oracle, m, n, seed):
    """Sec. 5.4: with two panels mCQR2GS can break down at kappa = 1e15; the
    smaller panel width is the paper's remedy.  Plain Alg. 9 reports a
    breakdown; the adaptive width finishes with O(u) orthogonality and
    residual, an upper triangular R with positive diagonal, and the panels
    before the rejected one untouched."""
    A = make_test_matrix(m, n, 1e15, seed)
    b = n // 2
    Qp, Rp, stp = oracle.mcqr2gs(A, b, check=False)
    assert stp > 0
    Q, R, bf = oracle.mcqr2gs_halving(A, b)
    assert bf < b and n % bf == 0
    assert orth_err(Q) < 1e-13 and resid(A, Q, R) < 1e-14
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    U1, st1 = oracle.chol(oracle.gram(A[:, :b]))  # the rule on panel 1, from the oracle's own factor
    d = np.diag(U1)
    if st1 == 0 and (d.max() / d.min()) ** 2 <= U_RULE:  # rejected at panel 2: panel 1 is plain Alg. 9's
        assert np.array_equal(Q[:, :b], Qp[:, :b]) and np.array_equal(R[:b, :b], Rp[:b, :b])


def test_halving_one_column_breakdown_is_reported(oracle):
    """A zero column can be cut down to a one-column panel but not further:
    the breakdown is reported with its global column."""
    A = make_test_matrix(1000, 8, 1e2, seed=23)
    A[:, 5] = 0.0
    _, _, bf, st = oracle.mcqr2gs_halving(A, 8, check=False)
    assert st == 6 and bf == 1
