"""Mutation test of the oracle's pins (CPU only).

Plausible mistakes -- a flipped sign, a dropped term, a wrong index, a
transposed operand, a factor product in the wrong order -- are planted in
copies of oracle/cqr_oracle.c, each copy is compiled on its own, and the pin
checks (the same facts test_oracle_pins.py uses: the exact dyadic QR,
Householder by brute force, the paper's accuracy targets, the breakdown
status, the closed form of the shifted CholeskyQR on orthonormal columns,
the runtime repetition rule on both sides of its threshold, torch autograd
for the adjoint) must reject every mutant.  The
unmutated source must pass them all.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from _helpers import exact_qr_case, load_exact_golden, orth_err, rel_diff, resid, sign_normalised_qr
from testmatrices import make_test_matrix

SRC = os.path.join(os.path.dirname(oracle.__file__), "cqr_oracle.c")

MUTATIONS = [
    ("gram: transposed operand index", "const double* yc = Y + c * ldy;", "const double* yc = Y + a * ldy;"),
    ("chol: sign of the diagonal update", "s -= AT(U, ldu, i, j) * AT(U, ldu, i, j);",
     "s += AT(U, ldu, i, j) * AT(U, ldu, i, j);"),
    ("chol: wrong row in the off-diagonal sum", "t -= AT(U, ldu, i, j) * AT(U, ldu, i, c);",
     "t -= AT(U, ldu, i, j) * AT(U, ldu, j, c);"),
    ("chol: no breakdown check", "if (!(s > 0.0) || !isfinite(s)) return (int)(j + 1);", "if (0) return 1;"),
    ("trsm: dropped first term", "      for (i64 i = 0; i < c; ++i) {\n        const double* qi = X + i * ldx;",
     "      for (i64 i = 1; i < c; ++i) {\n        const double* qi = X + i * ldx;"),
    ("update: wrong sign", "for (i64 r = r0; r < r1; ++r) xc[r] = xc[r] - s[r - r0];",
     "for (i64 r = r0; r < r1; ++r) xc[r] = xc[r] + s[r - r0];"),
    ("cqr2: R1 R2 instead of R2 R1", "if (!st) small_mm(n, n, n, R2, n, 1, R1, n, 1, R, ldr);\n  free(R1);\n  free(R2);\n  return st;\n}\n\n/* Alg. 5",
     "if (!st) small_mm(n, n, n, R1, n, 1, R2, n, 1, R, ldr);\n  free(R1);\n  free(R2);\n  return st;\n}\n\n/* Alg. 5"),
    ("cqrgs: projection not applied", "      or_update(m, b, w, Ar, ldx, Aj, ldx, Yp, ldr);\n    }\n  }\n  return 0;",
     "      (void)Ar;\n    }\n  }\n  return 0;"),
    ("cqr2gs: second pass skipped", "  if (!st) st = or_cqrgs(m, n, b, X, ldx, R2, n);",
     "  if (!st) { for (i64 i = 0; i < n * n; ++i) R2[i] = (i % (n + 1)) == 0; }"),
    ("mcqr2gs: projection against the current panel", "    double* Qprev = X + (j - 1) * b * ldx;",
     "    double* Qprev = X + (j > 1 ? j - 2 : 0) * b * ldx;"),
    ("mcqr2gs: re-orthogonalisation dropped", "    or_update(m, jb, b, Aj, ldx, X, ldx, Z, jb);\n",
     "    (void)Z;\n"),
    ("mcqr2gs: S1 S2 instead of S2 S1", "small_mm(b, b, b, S2, b, 1, S1, b, 1, &AT(R, ldr, jb, jb), ldr);",
     "small_mm(b, b, b, S1, b, 1, S2, b, 1, &AT(R, ldr, jb, jb), ldr);"),
    ("mcqr2gs: Y not recorded in R", "    or_update(m, b, w, Aj, ldx, Qprev, ldx, Yp, ldr);\n    st = or_cqr(m, b, Aj, ldx, S1, b);",
     "    or_update(m, b, w, Aj, ldx, Qprev, ldx, Yp, ldr);\n    for (i64 c = 0; c < w; ++c) for (i64 r = 0; r < b; ++r) Yp[r + c * ldr] = 0.0;\n    st = or_cqr(m, b, Aj, ldx, S1, b);"),
    ("backward: copyltu copies the upper triangle", "    for (i64 a = 0; a < c; ++a) M[a + c * n] = M[c + a * n];",
     "    for (i64 a = 0; a < c; ++a) M[c + a * n] = M[a + c * n];"),
    ("backward: sign of Qbar^T Q", "      M[a + c * n] = s - G[a + c * n];", "      M[a + c * n] = s + G[a + c * n];"),
    ("backward: R instead of R^T in the final solve", "        double u = AT(R, ldr, c, i);\n        for (i64 r = r0; r < r1; ++r) s[r - r0] -= ai[r] * u;",
     "        double u = AT(R, ldr, i, c);\n        for (i64 r = r0; r < r1; ++r) s[r - r0] -= ai[r] * u;"),
    ("householder: no sign normalisation", "    if (AT(R, ldr, j, j) < 0.0) {", "    if (0) {"),
    ("scqr: shift subtracted", "for (i64 j = 0; j < b; ++j) W[j + j * b] += s;",
     "for (i64 j = 0; j < b; ++j) W[j + j * b] -= s;"),
    ("scqr: shift without sqrt(m)", "double s = sqrt((double)m) * ldexp(1.0, -53) * fro2;",
     "double s = ldexp(1.0, -53) * fro2;"),
    ("scqr3: one CholeskyQR after the shifted pass", "  if (!st) st = or_cqr2(m, n, X, ldx, R2, n);",
     "  if (!st) st = or_cqr(m, n, X, ldx, R2, n);"),
    ("adaptive: threshold too loose", "const double tau = 8.0 * ldexp(1.0, -53);", "const double tau = ldexp(1.0, -20);"),
    ("adaptive: never fires", "const double tau = 8.0 * ldexp(1.0, -53);", "const double tau = 0.0;"),
    ("halving: breakdown not rejected", "  if (chol_status) return 1;\n", "  if (chol_status) return 0;\n"),
    ("halving: bound without the factor 64", "return dmax * dmax * 64.0 * ldexp(1.0, -53) > dmin * dmin;",
     "return dmax * dmax * ldexp(1.0, -53) > dmin * dmin;"),
    ("halving: bound 16x tighter", "return dmax * dmax * 64.0 * ldexp(1.0, -53) > dmin * dmin;",
     "return dmax * dmax * 1024.0 * ldexp(1.0, -53) > dmin * dmin;"),
    ("halving: Z S1 term dropped", "        for (i64 a = 0; a < c0; ++a) AT(R, ldr, a, c0 + c) += ZS[a + c * c0];",
     "        for (i64 a = 0; a < c0; ++a) AT(R, ldr, a, c0 + c) += 0.0 * ZS[a + c * c0];"),
]


def _pins(o) -> dict:
    """Run the pin checks through the currently routed oracle; True = passes."""
    res = {}

    def check(name, fn):
        try:
            res[name] = bool(fn())
        except Exception:
            res[name] = False

    A, Q0, R0 = load_exact_golden()

    def exact():
        for f in (lambda X, b: o.mcqr2gs(X, b), lambda X, b: o.cqr2gs(X, b), lambda X, b: o.cqr2(X)):
            for b in (2, 4, 8):
                Q, R = f(A, b)
                if not (np.array_equal(Q, Q0) and np.array_equal(R, R0)):
                    return False
        return True

    check("exact_golden", exact)

    def brute():
        X = make_test_matrix(33, 6, 1e3, seed=5)
        Qn, Rn = sign_normalised_qr(X)
        Qh, Rh = o.householder(X)
        ok = rel_diff(Rh, Rn) < 1e-12
        for f in (o.mcqr2gs, o.cqr2gs):
            for b in (2, 3, 6):
                Q, R = f(X, b)
                ok = ok and rel_diff(R, Rn) < 1e-10 and np.abs(Q - Qn).max() < 1e-10
        return ok

    check("brute_force", brute)

    def accuracy():
        X = make_test_matrix(2000, 40, 1e12, seed=6)
        ok = True
        for f, b in ((o.mcqr2gs, 10), (o.cqr2gs, 4)):
            Q, R = f(X, b)
            ok = ok and orth_err(Q) < 1e-13 and resid(X, Q, R) < 1e-14
            ok = ok and np.all(np.diag(R) > 0) and np.all(np.tril(R, -1) == 0)
        return ok

    check("accuracy", accuracy)

    def breakdown():
        _, st = o.chol(np.diag([4.0, 1.0, -1.0, 2.0]))
        return st == 3

    check("breakdown", breakdown)

    def shifted():
        # Alg. 4 on exactly orthonormal columns: W = I, s = sqrt(m) u n, R = sqrt(1 + s) I, Q = A / sqrt(1 + s)
        _, Qo, _ = exact_qr_case(4096, 16, seed=11)
        d = np.sqrt(1.0 + np.sqrt(4096.0) * 2.0 ** -53 * 16)
        Q1, R1 = o.scqr(Qo)
        ok = np.array_equal(R1, d * np.eye(16)) and np.array_equal(Q1, Qo / d)
        X = make_test_matrix(2000, 30, 1e12, seed=9)
        Q, R = o.scqr3(X)
        return ok and orth_err(Q) < 1e-13 and resid(X, Q, R) < 1e-14 and np.all(np.diag(R) > 0)

    check("shifted", shifted)

    def adaptive():
        # silent where the second pass matters (kappa = 1e4), fires on orthonormal panels (kappa = 1)
        X = make_test_matrix(3000, 48, 1e4, seed=12)
        Qd, Rd = o.mcqr2gs(X, 16)
        Qa, Ra = o.mcqr2gs(X, 16, adaptive=True)
        ok = np.array_equal(Qd, Qa) and np.array_equal(Rd, Ra)
        X = make_test_matrix(3000, 48, 1.0, seed=13)
        Qd, Rd = o.mcqr2gs(X, 16)
        Qa, Ra = o.mcqr2gs(X, 16, adaptive=True)
        return ok and not np.array_equal(Qd, Qa) and orth_err(Qa) < 1e-14 and resid(X, Qa, Ra) < 1e-15

    check("adaptive", adaptive)

    def adjoint():
        import torch

        m, n = 50, 6
        X = make_test_matrix(m, n, 1e2, seed=7)
        rng = np.random.default_rng(8)
        dQ = rng.standard_normal((m, n))
        dR = np.triu(rng.standard_normal((n, n)))
        At = torch.tensor(X, requires_grad=True)
        Qt, Rt = torch.linalg.qr(At)
        D = torch.sign(torch.diagonal(Rt)).detach()
        ((Qt * D * torch.tensor(dQ)).sum() + (Rt * D[:, None] * torch.tensor(dR)).sum()).backward()
        Q, R = o.mcqr2gs(X, 3)
        return rel_diff(o.backward(Q, R, dQ, dR), At.grad.numpy()) < 1e-10

    check("adjoint", adjoint)

    def halving():
        # no rejection: Alg. 9 itself (ratio at 0.35 of the bound)
        X = make_test_matrix(2000, 40, 1e15, seed=1)
        Q, R, bf = o.mcqr2gs_halving(X, 20)
        Q0, R0 = o.mcqr2gs(X, 20)
        ok = bf == 20 and np.array_equal(Q, Q0) and np.array_equal(R, R0)
        # first panel rejected by the ratio alone (10x over the bound): Alg. 9 with b = 10
        X = make_test_matrix(2000, 40, 1e15, seed=8)
        Q, R, bf = o.mcqr2gs_halving(X, 20)
        Q0, R0 = o.mcqr2gs(X, 10)
        ok = ok and bf == 10 and np.array_equal(Q, Q0) and np.array_equal(R, R0)
        # two-panel breakdowns recovered to O(u)
        for m, n, seed in ((2000, 40, 2), (4000, 80, 6)):
            X = make_test_matrix(m, n, 1e15, seed)
            Q, R, bf, st = o.mcqr2gs_halving(X, n // 2, check=False)
            ok = ok and st == 0 and bf < n // 2 and orth_err(Q) < 1e-13 and resid(X, Q, R) < 1e-14
        return ok

    check("halving", halving)
    return res


def _build_mutant(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    lib = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11", str(src),
                           "-o", str(lib), "-lm"])
    return oracle.open_library(str(lib))


def test_unmutated_oracle_passes_all_pins():
    res = _pins(oracle)
    assert all(res.values()), res


@pytest.mark.parametrize("desc,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutant_is_rejected(tmp_path, desc, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor not unique/present: {desc}"
    lib = _build_mutant(tmp_path, "mutant", text.replace(old, new))
    with oracle.using_library(lib):
        res = _pins(oracle)
    assert not all(res.values()), f"mutation survived the pins: {desc}"
