"""Phase ranges of the enqueue (NVTX domain "cqr" and cqr_set_trace).

The phases must follow the steps of the algorithm they bracket: Alg. 9's
step 1 on the first panel, then per panel j >= 1 the projection and
update (steps 3-5), the CholeskyQR (step 6), the re-orthogonalisation
(step 7), the second CholeskyQR (step 8) and the R products; Alg. 7 as two
passes of Alg. 6 with a CholeskyQR and a projection/update per panel.  Each
range closes before the next opens.
"""
import numpy as np
import pytest

from testmatrices import make_test_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(A):
    return torch.from_numpy(np.asfortranarray(A)).cuda().t().contiguous().t()


def well_nested(events):
    stack = []
    for name, panel, begin in events:
        if begin:
            stack.append((name, panel))
        else:
            assert stack and stack[-1] == (name, panel), (name, panel, stack)
            stack.pop()
    return not stack


def test_mcqr2gs_phases(cuda_lib):
    P = cuda_lib
    A = dev(make_test_matrix(4000, 96, 1e6, seed=1))
    with P.PhaseTrace() as t:
        P.factor(A, 32, "mcqr2gs")
    expect = [("cqr2_first_panel", 0)]
    for j in (1, 2):
        expect += [("project_update", j), ("cqr", j), ("reorthogonalise", j), ("cqr_final", j), ("r_update", j)]
    assert t.phases() == expect
    assert well_nested(t.events)


def test_cqr2gs_and_whole_matrix_phases(cuda_lib):
    P = cuda_lib
    A = dev(make_test_matrix(4000, 64, 1e6, seed=2))
    with P.PhaseTrace() as t:
        P.factor(A, 32, "cqr2gs")
    one_pass = [("cqr", 0), ("project_update", 0), ("cqr", 1)]
    assert t.phases() == [("cqrgs_pass", 0)] + one_pass + [("cqrgs_pass", 1)] + one_pass + [("r_update", -1)]
    assert well_nested(t.events)
    for variant in ("cqr2", "scqr3"):
        with P.PhaseTrace() as t:
            P.factor(A, 0, variant)
        assert t.phases() == [(variant, -1)] and well_nested(t.events)


def test_halving_phases_name_the_first_column(cuda_lib):
    """With the adaptive width a rejected first panel shows two panel tests
    at column 0; later panels are named by their first column."""
    P = cuda_lib
    A = dev(make_test_matrix(5000, 64, 1e13, seed=1))  # the 64-column panel is rejected, b -> 32
    info = {}
    with P.PhaseTrace() as t:
        P.factor(A, 64, "mcqr2gs", halving=True, info=info)
    assert info["panel_b"] == 32
    ph = t.phases()
    assert ph[:2] == [("panel_test", 0), ("panel_test", 0)]
    assert ("project_update", 32) in ph and ("reorthogonalise", 32) in ph and ("r_update", 32) in ph
    assert well_nested(t.events)


def test_tracing_off_after_the_context(cuda_lib):
    P = cuda_lib
    A = dev(make_test_matrix(2000, 32, 1e3, seed=3))
    with P.PhaseTrace() as t:
        pass
    P.factor(A, 16)
    assert t.events == []
