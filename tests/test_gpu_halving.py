"""Adaptive panel width (CQR_HALVE) on the GPU against the oracle's rule
(or_mcqr2gs_halving, pinned in tests/test_oracle_pins.py).

The inputs are chosen so that every panel decision is far from the bound
(1/(64 u) on the squared diagonal ratio of the first Cholesky factor): a
rejected panel's Gram matrix is numerically singular by orders of magnitude
(the whole 64- or 128-column matrix at kappa >= 1e13) or, for 5000 x 64 at
kappa = 1e15 (seed 5), its 32-column half breaks down in the oracle and has
a ratio 15x over the bound in LAPACK; every accepted panel is at least 10x
below it.  So both sides must take the same decisions:
  * the final width equals the oracle's;
  * the panels were rejected only at the first panel, so the result must
    equal, bit for bit, the GPU's plain mCQR2GS at the final width (the
    rejected attempts leave the panel untouched);
  * orthogonality and residual meet the bounds; with no rejection
    (kappa = 1e5) the result is the fixed-width one and matches the oracle
    element-wise;
  * a zero column is cut down to a one-column panel and its breakdown is
    reported at the oracle's column.
"""
import numpy as np
import pytest

from _helpers import orth_err, rel_diff, resid
from testmatrices import make_test_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu(P, A, b, **kw):
    At = P.colmajor(torch.from_numpy(np.asfortranarray(A)).cuda())
    info = {}
    Q, R = P.factor(At, b, "mcqr2gs", info=info, **kw)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), R.cpu().numpy(), info.get("panel_b")


@pytest.mark.parametrize("m,n,kappa,b,seed,b_final", [
    (5000, 64, 1e13, 64, 1, 32), (5000, 64, 1e13, 64, 2, 32), (5000, 64, 1e15, 64, 5, 16),
    (6000, 128, 1e14, 128, 1, 64), (8000, 64, 1e12, 64, 3, 32)])
def test_halving_matches_the_oracle_rule(cuda_lib, oracle, m, n, kappa, b, seed, b_final):
    P = cuda_lib
    A = make_test_matrix(m, n, kappa, seed)
    Qo, Ro, bo = oracle.mcqr2gs_halving(A, b)
    assert bo == b_final
    Qg, Rg, bg = gpu(P, A, b, halving=True)
    assert bg == bo
    assert orth_err(Qg) <= 1e-13 and resid(A, Qg, Rg) <= 1e-14
    assert np.all(np.tril(Rg, -1) == 0) and np.all(np.diag(Rg) > 0)
    Qf, Rf, _ = gpu(P, A, bg)  # plain mCQR2GS at the final width
    assert np.array_equal(Qg, Qf) and np.array_equal(Rg, Rf)


def test_halving_without_rejection_is_the_fixed_width(cuda_lib, oracle):
    P = cuda_lib
    A = make_test_matrix(20000, 64, 1e5, seed=6300)
    Qg, Rg, bg = gpu(P, A, 16, halving=True)
    Qf, Rf, _ = gpu(P, A, 16)
    assert bg == 16 and np.array_equal(Qg, Qf) and np.array_equal(Rg, Rf)
    Qo, Ro, bo = oracle.mcqr2gs_halving(A, 16)
    assert bo == 16 and rel_diff(Rg, Ro) <= 1e-11 and np.abs(Qg - Qo).max() <= 1e-11


def test_halving_reports_a_zero_column(cuda_lib, oracle):
    P = cuda_lib
    A = make_test_matrix(1000, 8, 1e2, seed=23)
    A[:, 5] = 0.0
    _, _, bo, st = oracle.mcqr2gs_halving(A, 8, check=False)
    assert st == 6 and bo == 1
    with pytest.raises(P.CQRError) as ei:
        gpu(P, A, 8, halving=True)
    assert ei.value.code == st
