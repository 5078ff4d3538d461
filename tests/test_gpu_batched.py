"""Batched factorisation.

Stream-pool schedule: every member equals the single-call result bit for bit
(same sizes, same panel width, same deterministic reduction order) and
matches the oracle within the parity tolerances.

Persistent schedule (one cooperative launch, groups of CTAs per matrix):
every member matches the oracle within the parity tolerances (element-wise
for kappa <= 1e6, norms up to 1e15), runs are bitwise reproducible, a
captured CUDA graph replays bitwise the eager result, statuses are per
matrix, every group size gives the same accuracy, the on-device adaptive
width takes the oracle's decisions, and a group-barrier wait that expires
leaves CQR_STATUS_TIMEOUT and a usable context.
"""
import numpy as np
import pytest

from _helpers import orth_err, rel_diff, resid
from testmatrices import batch_specs, make_test_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORTH_TOL, RES_TOL, R_TOL, Q_TOL = 1e-13, 1e-14, 1e-11, 1e-11


def _t(x):
    return torch.from_numpy(np.asfortranarray(x)).cuda()


def _panel_for(n, kappa):
    # enough panels for the condition number (3 at 1e15, Sec. 5.4)
    k = 1 if kappa < 1e7 else (2 if kappa < 1e11 else 4)
    while n % k:
        k += 1
    return n // k


def _check_against_oracle(oracle, A, Qb, Rb, b, kappa, variant="mcqr2gs"):
    Qn, Rn = Qb.cpu().numpy(), Rb.cpu().numpy()
    assert np.all(np.tril(Rn, -1) == 0) and np.all(np.diag(Rn) > 0)
    assert orth_err(Qn) < ORTH_TOL and resid(A, Qn, Rn) < RES_TOL
    if kappa <= 1e6:
        Qo, Ro = (oracle.mcqr2gs if variant == "mcqr2gs" else oracle.cqr2gs)(A, b)
        assert rel_diff(Rn, Ro) < R_TOL and np.abs(Qn - Qo).max() < Q_TOL


# --------------------------------------------------------------------------- stream pool: bitwise = single calls
@pytest.mark.parametrize("variant", ["mcqr2gs", "cqr2gs"])
def test_batched_pool_equals_single(cuda_lib, oracle, variant):
    P = cuda_lib
    specs = batch_specs(count=24, m_range=(200, 30000))
    As = [make_test_matrix(m, n, k, s) for (m, n, k, s) in specs]
    bs = [_panel_for(n, k) for (m, n, k, s) in specs]
    if variant == "cqr2gs":  # CQR2GS needs narrower panels at high kappa (Sec. 5.3)
        bs = [max(1, n // 8) if k > 1e7 else b for b, (m, n, k, s) in zip(bs, specs)]
    res = P.factor_batched([_t(A) for A in As], bs, variant, schedule="pool")
    for i, ((Qb, Rb), A, b, spec) in enumerate(zip(res, As, bs, specs)):
        Qs, Rs = P.factor(_t(A), b, variant)
        assert torch.equal(Qb, Qs) and torch.equal(Rb, Rs), i
        _check_against_oracle(oracle, A, Qb, Rb, b, spec[2], variant)


def test_batched_pool_status_per_matrix(cuda_lib):
    P = cuda_lib
    A1 = make_test_matrix(3000, 16, 1e2, seed=2100)
    A2 = make_test_matrix(4000, 16, 1e2, seed=2101)
    A2[:, 7] = 0.0
    A3 = make_test_matrix(5000, 32, 1e2, seed=2102)
    status = torch.zeros(3, dtype=torch.int32, device="cuda")
    P.factor_batched([_t(A1), _t(A2), _t(A3)], [4, 4, 8], check=False, status=status, schedule="pool")
    torch.cuda.synchronize()
    assert status.tolist() == [0, 8, 0]


def test_batched_pool_graph_replay(cuda_lib):
    """The pool schedule captured into a CUDA graph gives the same bits as
    the single calls, and replays on refilled inputs."""
    P = cuda_lib
    specs = batch_specs(count=12, m_range=(500, 20000), seed=4100)
    As = [_t(make_test_matrix(m, n, k, s)) for (m, n, k, s) in specs]
    bs = [_panel_for(n, k) for (m, n, k, s) in specs]
    g = P.BatchedGraph(As, bs, schedule="pool")
    out = g.replay()
    torch.cuda.synchronize()
    assert int((g.status != 0).sum()) == 0
    for (Qg, Rg), A, b in zip(out, As, bs):
        Qs, Rs = P.factor(A, b)
        assert torch.equal(Qg, Qs) and torch.equal(Rg, Rs)
    new = [make_test_matrix(m, n, k, s + 1000) for (m, n, k, s) in specs]
    for A, An in zip(As, new):
        A.copy_(torch.from_numpy(An))
    out = g.replay()
    torch.cuda.synchronize()
    for (Qg, Rg), A, b in zip(out, As, bs):
        Qs, Rs = P.factor(A, b)
        assert torch.equal(Qg, Qs) and torch.equal(Rg, Rs)


def test_batched_empty(cuda_lib):
    assert cuda_lib.factor_batched([]) == []


# --------------------------------------------------------------------------- persistent launch
def _persistent_batch(count=40, seed=4200, m_range=(200, 40000)):
    specs = batch_specs(count=count, m_range=m_range, seed=seed)
    As = [make_test_matrix(m, n, k, s) for (m, n, k, s) in specs]
    bs = [_panel_for(n, k) for (m, n, k, s) in specs]
    return specs, As, bs


def test_persistent_matches_oracle(cuda_lib, oracle):
    P = cuda_lib
    specs, As, bs = _persistent_batch()
    res = P.factor_batched([_t(A) for A in As], bs)
    for (Qb, Rb), A, b, spec in zip(res, As, bs, specs):
        _check_against_oracle(oracle, A, Qb, Rb, b, spec[2])


def test_persistent_in_place_and_ragged_rows(cuda_lib, oracle):
    """In place (Q_i = A_i) and row counts that are no multiple of the row
    sub-block or of the group size, including m_i < 64 and m_i == n_i."""
    P = cuda_lib
    shapes = [(1000, 16, 4), (99, 32, 8), (64, 64, 16), (130, 128, 32), (12345, 128, 64), (4097, 48, 12)]
    As = [make_test_matrix(m, n, 1e4, seed=4300 + i) for i, (m, n, b) in enumerate(shapes)]
    Ts = [_t(A) for A in As]
    res = P.factor_batched(Ts, [b for (m, n, b) in shapes], inplace=True)
    for (Qb, Rb), T, A, (m, n, b) in zip(res, Ts, As, shapes):
        assert Qb.data_ptr() == T.data_ptr()
        _check_against_oracle(oracle, A, Qb, Rb, b, 1e4)


def test_persistent_is_deterministic(cuda_lib):
    P = cuda_lib
    specs, As, bs = _persistent_batch(count=30, seed=4210)
    Ts = [_t(A) for A in As]
    r1 = P.factor_batched(Ts, bs)
    r2 = P.factor_batched(Ts, bs)
    for (Q1, R1), (Q2, R2) in zip(r1, r2):
        assert torch.equal(Q1, Q2) and torch.equal(R1, R2)


@pytest.mark.parametrize("group", [1, 2, 4, 8, 19])
def test_persistent_group_sizes(cuda_lib, oracle, group):
    P = cuda_lib
    specs, As, bs = _persistent_batch(count=20, seed=4220 + group)
    res = P.factor_batched([_t(A) for A in As], bs, group=group)
    for (Qb, Rb), A, b, spec in zip(res, As, bs, specs):
        _check_against_oracle(oracle, A, Qb, Rb, b, spec[2])


def test_persistent_status_per_matrix(cuda_lib, oracle):
    P = cuda_lib
    A1 = make_test_matrix(3000, 16, 1e2, seed=2100)
    A2 = make_test_matrix(4000, 16, 1e2, seed=2101)
    A2[:, 7] = 0.0
    A3 = make_test_matrix(5000, 32, 1e2, seed=2102)
    status = torch.full((3,), -7, dtype=torch.int32, device="cuda")
    res = P.factor_batched([_t(A1), _t(A2), _t(A3)], [4, 4, 8], check=False, status=status)
    torch.cuda.synchronize()
    _, _, st_o = oracle.mcqr2gs(A2, 4, check=False)
    assert status.tolist() == [0, st_o, 0] and st_o == 8
    _check_against_oracle(oracle, A3, res[2][0], res[2][1], 8, 1e2)


def test_persistent_graph_replay(cuda_lib):
    P = cuda_lib
    specs, As, bs = _persistent_batch(count=16, seed=4230)
    Ts = [_t(A) for A in As]
    eager = P.factor_batched(Ts, bs)
    eager = [(Q.clone(), R.clone()) for Q, R in eager]
    g = P.BatchedGraph(Ts, bs)
    for _ in range(2):
        out = g.replay()
        torch.cuda.synchronize()
        assert int((g.status != 0).sum()) == 0
        for (Qg, Rg), (Qe, Re) in zip(out, eager):
            assert torch.equal(Qg, Qe) and torch.equal(Rg, Re)


@pytest.mark.parametrize("m,n,kappa,seed,b_final", [(5000, 64, 1e13, 1, 32), (5000, 64, 1e15, 5, 16),
                                                    (6000, 128, 1e14, 1, 64), (8000, 64, 1e12, 3, 32)])
def test_persistent_halving_matches_oracle_rule(cuda_lib, oracle, m, n, kappa, seed, b_final):
    """Adaptive width on the device, starting from one panel (b = n): the
    decisions are far from the bound on these inputs (see test_gpu_halving)."""
    P = cuda_lib
    A = make_test_matrix(m, n, kappa, seed)
    W = make_test_matrix(20000, 32, 1e3, seed + 50)  # a well-conditioned neighbour in the same launch
    ws = torch.empty(P.batched_workspace_size([m, 20000], [n, 32], [n, 32], halving=True), dtype=torch.uint8,
                     device="cuda")
    res = P.factor_batched([_t(A), _t(W)], [n, 32], workspace=ws, halving=True)
    _, _, bo = oracle.mcqr2gs_halving(A, n)
    assert bo == b_final
    assert P.batched_panel_widths(ws, 2) == [b_final, 32]
    Qn, Rn = res[0][0].cpu().numpy(), res[0][1].cpu().numpy()
    assert orth_err(Qn) < ORTH_TOL and resid(A, Qn, Rn) < RES_TOL
    _check_against_oracle(oracle, W, res[1][0], res[1][1], 32, 1e3)


def test_persistent_barrier_expiry(cuda_lib):
    """One CTA of group 0 skips a group-barrier arrival (test hook, 1 ms
    bound): the launch returns, unfinished matrices read CQR_STATUS_TIMEOUT,
    and the next launch on the same context succeeds."""
    P = cuda_lib
    L = P.load()
    specs, As, bs = _persistent_batch(count=24, seed=4240)
    Ts = [_t(A) for A in As]
    status = torch.zeros(len(Ts), dtype=torch.int32, device="cuda")
    assert L.cqr_test_arm_barrier_expiry(0, 1, 2, 1_000_000) == 0
    try:
        P.factor_batched(Ts, bs, check=False, status=status)
        torch.cuda.synchronize()
    finally:
        L.cqr_test_arm_barrier_expiry(-1, 0, 1, 1)
    st = status.tolist()
    assert P._capi.STATUS_TIMEOUT in st
    assert all(s in (0, P._capi.STATUS_TIMEOUT) for s in st)
    res = P.factor_batched(Ts, bs)  # raises on any nonzero status
    for (Qb, Rb), A in zip(res, As):
        assert orth_err(Qb.cpu().numpy()) < ORTH_TOL
