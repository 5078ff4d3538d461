"""Host-side logic of the C ABI and the autotuner, without a GPU.

Every call below fails argument validation before the library makes its
first CUDA call, so the pointers passed are never dereferenced and nothing
is launched: the tests run on a machine without a GPU (and would run
unchanged on one).  They pin the LAPACK-style argument codes that
include/cqr.h documents, the workspace sizing rules and the autotuner's
stability filter (minimum panel counts of Sec. 5.3 / Sec. 5.4).
"""
import ctypes

import pytest

import paper_2405_04237_gb300 as P
from paper_2405_04237_gb300 import _capi
from paper_2405_04237_gb300.autotune import candidates, min_panels

MC, CG, C2, S3 = _capi.MCQR2GS, _capi.CQR2GS, _capi.CQR2, _capi.SCQR3

# Fake, 256-byte aligned device addresses far apart (never dereferenced).
A_ADDR, Q_ADDR, R_ADDR, W_ADDR, S_ADDR = (0x7F0000000000 + (i << 36) for i in range(5))


def vp(x):
    return ctypes.c_void_p(x)


@pytest.fixture(scope="module")
def L():
    return P.load()


def factor_rc(L, m=1000, n=64, A=A_ADDR, lda=None, b=16, Q=Q_ADDR, ldq=None, R=R_ADDR, ldr=None, variant=MC,
              ws=W_ADDR, ws_bytes=None):
    lda = m if lda is None else lda
    ldq = m if ldq is None else ldq
    ldr = n if ldr is None else ldr
    if ws_bytes is None:
        ws_bytes = 1 << 40
    return L.cqr_factor(m, n, vp(A), lda, b, vp(Q), ldq, vp(R), ldr, variant, vp(ws), ws_bytes, vp(0))


def test_factor_argument_codes(L):
    assert factor_rc(L, m=10, n=16) == -1                      # m < n
    assert factor_rc(L, m=0, n=0) == -1                        # m < 1
    assert factor_rc(L, n=0) == -2                             # n < 1
    assert factor_rc(L, A=0) == -3                             # A null
    assert factor_rc(L, lda=999) == -4                         # lda < m
    assert factor_rc(L, b=5) == -5                             # b does not divide n
    assert factor_rc(L, b=-1) == -5                            # negative panel width
    assert factor_rc(L, m=4096, n=1024, b=1024) == -5          # b above CQR_MAX_PANEL
    assert factor_rc(L, m=9000, n=1024, variant=C2) == -2      # CholeskyQR2: one panel, n <= CQR_MAX_PANEL
    assert factor_rc(L, m=9000, n=1024, variant=S3) == -2      # shifted CholeskyQR3 likewise
    assert factor_rc(L, Q=0) == -6                             # Q null
    assert factor_rc(L, Q=A_ADDR + 8 * 100) == -6              # Q overlaps A
    assert factor_rc(L, ldq=999) == -7                         # ldq < m
    assert factor_rc(L, Q=A_ADDR, lda=1000, ldq=1024) == -7    # in place with ldq != lda
    assert factor_rc(L, R=0) == -8                             # R null
    assert factor_rc(L, ldr=63) == -9                          # ldr < n
    assert factor_rc(L, variant=4) == -10                      # unknown variant
    assert factor_rc(L, variant=CG | _capi.EMULATED) == -10    # emulation is mCQR2GS only
    assert factor_rc(L, variant=CG | _capi.ADAPTIVE) == -10    # adaptive repetitions are mCQR2GS only
    assert factor_rc(L, variant=CG | _capi.HALVE) == -10       # adaptive panel width: mCQR2GS only
    assert factor_rc(L, variant=MC | _capi.HALVE | _capi.EMULATED) == -10
    assert factor_rc(L, variant=MC | _capi.HALVE | _capi.LOOKAHEAD) == -10
    assert factor_rc(L, ws=0) == -11                           # workspace null
    assert factor_rc(L, ws=W_ADDR + 8) == -11                  # workspace not 256-byte aligned
    need = L.cqr_workspace_size(1000, 64, 16, MC)
    assert need > 0
    assert factor_rc(L, ws_bytes=need - 1) == -12              # workspace too small


def factor_host_rc(L, m=1000, n=64, A=A_ADDR, lda=None, b=16, Q=Q_ADDR, ldq=None, R=R_ADDR, ldr=None, variant=MC,
                   Qd=S_ADDR, ldqd=None, Rd=W_ADDR + (1 << 35), ldrd=None, ws=W_ADDR, ws_bytes=1 << 40):
    lda = m if lda is None else lda
    ldq = m if ldq is None else ldq
    ldr = n if ldr is None else ldr
    ldqd = m if ldqd is None else ldqd
    ldrd = n if ldrd is None else ldrd
    return L.cqr_factor_host(m, n, vp(A), lda, b, vp(Q), ldq, vp(R), ldr, variant, vp(Qd), ldqd, vp(Rd), ldrd,
                             vp(ws), ws_bytes, vp(0))


def test_factor_host_argument_codes(L):
    """cqr_factor_host: the codes of cqr_factor for arguments 1-10 (host
    A, Q, R), then the device buffers Qd (13, 14) and Rd (15, 16)."""
    assert factor_host_rc(L, m=10, n=16) == -1
    assert factor_host_rc(L, n=0) == -2
    assert factor_host_rc(L, m=9000, n=1024, variant=C2) == -2
    assert factor_host_rc(L, A=0) == -3
    assert factor_host_rc(L, lda=999) == -4
    assert factor_host_rc(L, b=5) == -5
    assert factor_host_rc(L, Q=0) == -6
    assert factor_host_rc(L, Q=A_ADDR + 8 * 100) == -6          # host Q overlaps host A
    assert factor_host_rc(L, ldq=999) == -7
    assert factor_host_rc(L, Q=A_ADDR, lda=1000, ldq=1024) == -7  # in place on the host with ldq != lda
    assert factor_host_rc(L, R=0) == -8
    assert factor_host_rc(L, ldr=63) == -9
    assert factor_host_rc(L, variant=4) == -10
    assert factor_host_rc(L, variant=CG | _capi.HALVE) == -10
    assert factor_host_rc(L, variant=MC | _capi.HALVE | _capi.LOOKAHEAD) == -10
    assert factor_host_rc(L, Qd=0) == -13
    assert factor_host_rc(L, ldqd=999) == -14
    assert factor_host_rc(L, Rd=0) == -15
    assert factor_host_rc(L, Rd=S_ADDR + 8 * 5000) == -15        # Rd inside Qd
    assert factor_host_rc(L, Rd=S_ADDR - 8 * 100) == -15         # Rd's tail reaches into Qd
    assert factor_host_rc(L, ldrd=63) == -16
    assert factor_host_rc(L, ws=0) == -11                        # no registered allocator
    assert factor_host_rc(L, ws=W_ADDR + 8) == -11
    need = L.cqr_workspace_size(1000, 64, 16, MC)
    assert factor_host_rc(L, ws_bytes=need - 1) == -12


def test_halving_workspace_covers_every_width(L):
    """The adaptive width's workspace holds the partial sums of every width
    the chain b, b/2, ..., 1 can reach, so it is never smaller than the
    fixed-width workspace of any width on the chain."""
    for m, n, b in ((100000, 1024, 128), (20000, 96, 24), (5000, 64, 64)):
        need = L.cqr_workspace_size(m, n, b, MC | _capi.HALVE)
        w = b
        while True:
            assert need >= L.cqr_workspace_size(m, n, w, MC)
            if w == 1:
                break
            w = max(d for d in range(1, w // 2 + 1) if w % d == 0)
    assert L.cqr_workspace_size(1000, 64, 16, CG | _capi.HALVE) == 0


def test_workspace_sizes(L):
    # invalid sizes give 0
    assert L.cqr_workspace_size(10, 16, 4, MC) == 0
    assert L.cqr_workspace_size(100, 16, 5, MC) == 0
    assert L.cqr_workspace_size(100, 16, 4, 9) == 0
    assert L.cqr_workspace_size(100, 16, 4, CG | _capi.EMULATED) == 0
    assert L.cqr_workspace_size(1000, 600, 0, C2) == 0
    # every size is a multiple of 256 and grows with m
    prev = 0
    for m in (64, 1000, 4096, 100000, 1 << 23):
        for var in (MC, CG, C2, S3):
            s = L.cqr_workspace_size(m, 64, 16, var)
            assert s > 0 and s % 256 == 0, (m, var, s)
        s = L.cqr_workspace_size(m, 64, 16, MC)
        assert s >= prev
        prev = s
    # the emulated products need the digit planes on top
    assert L.cqr_workspace_size(1 << 20, 256, 64, MC | _capi.EMULATED) > L.cqr_workspace_size(1 << 20, 256, 64, MC)
    # CQR2GS and sCQR3 keep two n x n triangles (R1, R2) that mCQR2GS does not
    assert L.cqr_workspace_size(1 << 16, 256, 64, CG) >= L.cqr_workspace_size(1 << 16, 256, 64, MC)
    # panel_b = 0 resolves to the default panel
    assert L.cqr_workspace_size(5000, 96, 0, MC) == L.cqr_workspace_size(5000, 96, L.cqr_default_panel(96), MC)


def test_default_panel_rule(L):
    """The largest divisor of n that is <= min(256, ceil(n/3)): at least three
    panels (Sec. 5.4) and b | n (Alg. 6)."""
    for n in range(1, 1200):
        b = L.cqr_default_panel(n)
        cap = min(256, -(-n // 3))
        assert n % b == 0 and 1 <= b <= max(cap, 1)
        assert all(n % c for c in range(b + 1, cap + 1))
    assert L.cqr_default_panel(0) == 0


def test_backward_argument_codes(L):
    def rc(m=1000, n=64, Q=Q_ADDR, ldq=1000, R=R_ADDR, ldr=64, dQ=A_ADDR, lddq=1000, dR=S_ADDR, lddr=64,
           dA=W_ADDR, ldda=1000, ws=W_ADDR + (1 << 35), ws_bytes=1 << 40):
        return L.cqr_backward(m, n, vp(Q), ldq, vp(R), ldr, vp(dQ), lddq, vp(dR), lddr, vp(dA), ldda, vp(ws),
                              ws_bytes, vp(0))

    assert rc(m=10) == -1
    assert rc(n=0) == -2
    assert rc(Q=0) == -3
    assert rc(ldq=999) == -4
    assert rc(R=0) == -5
    assert rc(ldr=63) == -6
    assert rc(lddq=999) == -8
    assert rc(lddr=63) == -10
    assert rc(dA=0) == -11
    assert rc(ldda=999) == -12
    assert rc(dA=Q_ADDR + 8) == -11                            # dA overlaps Q
    assert rc(ws=0) == -13
    assert rc(ws=W_ADDR + (1 << 35) + 16) == -13
    assert rc(ws_bytes=L.cqr_backward_workspace_size(1000, 64) - 1) == -14
    assert L.cqr_backward_workspace_size(10, 64) == 0
    assert L.cqr_backward_workspace_size(1000, 64) % 256 == 0


def test_batched_argument_codes(L):
    B = 3
    i64 = ctypes.c_int64 * B
    ms, ns, lds = i64(5000, 3000, 800), i64(64, 32, 16), i64(5000, 3000, 800)
    bs = (ctypes.c_int * B)(16, 8, 4)
    ptrs = lambda base: (ctypes.c_void_p * B)(*[base + (i << 33) for i in range(B)])
    Ap, Qp, Rp = ptrs(A_ADDR), ptrs(Q_ADDR), ptrs(R_ADDR)
    need = L.cqr_batched_workspace_size(B, ms, ns, bs, MC)
    assert need > 0 and need % 256 == 0
    # the workspace holds one slice per stream: at least the largest single workspace
    assert need >= max(L.cqr_workspace_size(m, n, b, MC) for m, n, b in zip(ms, ns, bs))

    def rc(batch=B, ms=ms, ns=ns, lds=lds, bs=bs, Ap=Ap, Qp=Qp, Rp=Rp, var=MC, status=S_ADDR, ws=W_ADDR,
           ws_bytes=need):
        return L.cqr_factor_batched(batch, ms, ns, lds, bs, Ap, Qp, Rp, var, vp(status), vp(ws), ws_bytes, vp(0))

    assert rc(batch=-1) == -1
    assert rc(batch=0) == 0                                    # nothing to do, nothing launched
    assert rc(ms=None) == -2
    assert rc(ns=i64(64, 3001, 16)) == -2                      # m_i < n_i
    assert rc(lds=i64(5000, 2999, 800)) == -2                  # lda_i < m_i
    assert rc(bs=(ctypes.c_int * B)(16, 7, 4)) == -5           # b_i does not divide n_i
    assert rc(Ap=None) == -6
    assert rc(Qp=(ctypes.c_void_p * B)(Q_ADDR, A_ADDR + (1 << 33) + 8, Q_ADDR + (2 << 33))) == -7  # Q_1 overlaps A_1
    assert rc(var=C2) == -9                                    # batched: mCQR2GS and CQR2GS only
    assert rc(status=0) == -10
    assert rc(ws=W_ADDR + 64) == -11
    assert rc(ws_bytes=need - 1) == -12


def test_noalloc_argument_codes_and_limit(L):
    def rc(m=1000, n=64, b=16, variant=MC):
        return L.cqr_factor_noalloc(m, n, vp(A_ADDR), m, b, vp(Q_ADDR), m, vp(R_ADDR), n, variant, vp(S_ADDR), vp(0))

    assert rc(m=10) == -1
    assert rc(b=5) == -5
    assert rc(variant=MC | _capi.EMULATED) == -10              # no flags: the fixed scratch has no room for planes
    # too large for the fixed array: refused before any CUDA call
    m, n, b = 16384, 16384, 512  # the re-orthogonalisation coefficients Z alone need n * b * 8 = 64 MiB
    assert L.cqr_workspace_size(m, n, b, MC) > _capi.NOALLOC_SCRATCH_BYTES
    assert rc(m=m, n=n, b=b) == _capi.ERR_NOALLOC_TOO_LARGE
    assert "CQR_NOALLOC_SCRATCH_BYTES" in P.status_string(_capi.ERR_NOALLOC_TOO_LARGE)


def test_allocator_registration_codes(L):
    """cqr_set_allocator: both callbacks or neither; with none registered, a
    NULL workspace stays an argument error (nothing is allocated or run)."""
    null_a, null_f = _capi.ALLOC_FN(), _capi.FREE_FN()
    a = _capi.ALLOC_FN(lambda nbytes, stream, ctx: None)
    f = _capi.FREE_FN(lambda ptr, nbytes, stream, ctx: None)
    assert L.cqr_set_allocator(null_a, f, None) == -1
    assert L.cqr_set_allocator(a, null_f, None) == -2
    assert L.cqr_set_allocator(null_a, null_f, None) == 0
    assert factor_rc(L, ws=0) == -11
    assert L.cqr_backward(1000, 64, vp(Q_ADDR), 1000, vp(R_ADDR), 64, vp(0), 1000, vp(0), 64, vp(W_ADDR), 1000,
                          vp(0), 0, vp(0)) == -13
    assert "cqr_set_allocator" in P.status_string(_capi.ERR_ALLOC)


def test_wait_expiry_hook_codes(L):
    """The test hook of the bounded waits is host-side only: arming and
    disarming launch nothing; its arguments are checked."""
    assert L.cqr_test_arm_wait_expiry(2, 0, 1000) == -1
    assert L.cqr_test_arm_wait_expiry(0, -1, 1000) == -2
    assert L.cqr_test_arm_wait_expiry(0, 0, 0) == -3
    assert L.cqr_test_arm_wait_expiry(1, 0, 3_000_000_000) == -3      # beyond the production bound
    assert L.cqr_test_arm_wait_expiry(0, 1, 1_000_000) == 0
    assert L.cqr_test_arm_wait_expiry(-1, 0, 1) == 0                  # disarm


def test_status_strings():
    assert P.status_string(0) == "success"
    assert "breakdown" in P.status_string(17)
    assert "invalid" in P.status_string(-3)
    assert "CUDA" in P.status_string(_capi.ERR_CUDA)
    assert "wait" in P.status_string(_capi.STATUS_TIMEOUT)
    st = ctypes.c_int(5)
    assert P.load().cqr_read_status(vp(0), vp(0), ctypes.byref(st)) == -1 and st.value == 5


def test_autotuner_stability_filter():
    """Minimum panel counts: mCQR2GS 1 / 2 / 3 panels up to 1e7 / 1e11 /
    beyond (Sec. 5.4, Fig. 6); CQR2GS 1 / 4 / 10 (Sec. 5.3, Fig. 3); an
    unknown condition number takes the strictest floor."""
    assert [min_panels("mcqr2gs", k) for k in (1e3, 1e7, 1e8, 1e11, 1e12, None)] == [1, 1, 2, 2, 3, 3]
    assert [min_panels("cqr2gs", k) for k in (1e3, 1e8, 1e12, None)] == [1, 4, 10, 10]
    assert min_panels("cqr2", 1e15) == 1
    c = candidates(1024, "mcqr2gs", 1e15)
    assert c == [16, 32, 64, 128, 256]
    assert all(1024 % b == 0 and 1024 // b >= 3 for b in c)
    assert candidates(1024, "cqr2gs", 1e15) == [16, 32, 64]
    assert candidates(64, "mcqr2gs", 1e3) == [16, 32, 64]
    # narrow matrices: below the lower bound only b = n, else the widest stable divisor
    assert candidates(12, "mcqr2gs", 1e15) == [4]
    assert candidates(16, "mcqr2gs", 1e3) == [16]


def test_kernel_class_names_match_the_binding(L):
    names = [L.cqr_kernel_class_name(i).decode() for i in range(len(_capi.KERNEL_CLASSES))]
    assert names == _capi.KERNEL_CLASSES
    assert L.cqr_launch_count() >= 0
