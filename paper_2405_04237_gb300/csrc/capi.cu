// Host driver and C ABI: the panel loops of mCQR2GS (Alg. 9), CQR2GS
// (Alg. 6 + Alg. 7), CholeskyQR2 (Alg. 3) and shifted CholeskyQR3 (Alg. 4 +
// Alg. 5), and the adjoint of A = QR.  Every step is a kernel launch on the
// caller's stream; nothing here computes on the host, allocates, or waits.
#include <string.h>

#include <mutex>
#include <vector>

#include "cqr.h"
#include "cqr_common.cuh"

using namespace cqr;

namespace {

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t status, skip, panel, W, S1, S2, rinv, Z, R1, R2, part, oz, total;
};

// Substitution block width of the emulated variant: its coupling products
// run on the tensor cores, so narrower blocks move FP64 substitution work
// (b * blk per row) into them.
constexpr int kTrsmEmuB = 32;

// Offsets of the words cqr_read_status and cqr_read_panel_width read.
constexpr size_t kStatusOffset = 0, kPanelOffset = 512;

// Panel width after a rejected panel (adaptive width): the largest divisor
// of b that is <= b/2, so that it still divides the remaining width.
int halved_width(int b) {
  for (int d = b / 2; d > 1; --d)
    if (b % d == 0) return d;
  return 1;
}

// Workspace plan.  The status word sits at offset 0 (cqr_read_status).
Layout make_layout(i64 m, i64 n, int b, int variant, bool emulated = false, bool halving = false) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const bool whole = (variant == CQR_CQR2 || variant == CQR_SCQR3);
  const i64 pw = whole ? n : b;  // panel width of every CQR
  L.status = take(sizeof(int));
  L.skip = take(sizeof(int));
  L.panel = take(sizeof(int));  // == kPanelOffset: every entry is 256-byte aligned
  L.W = take(sizeof(double) * pw * pw);
  L.S1 = take(sizeof(double) * pw * pw);
  L.S2 = take(sizeof(double) * pw * pw);
  L.rinv = take(sizeof(double) * pw);
  L.Z = take(variant == CQR_MCQR2GS ? sizeof(double) * n * b : 0);
  L.R1 = take((variant == CQR_CQR2GS || variant == CQR_SCQR3) ? sizeof(double) * n * n : 0);
  L.R2 = take((variant == CQR_CQR2GS || variant == CQR_SCQR3) ? sizeof(double) * n * n : 0);
  size_t pd = tn_partial_doubles(m, (int)pw, (int)pw, 1);
  if (!whole) {
    for (i64 j = 0; j * b < n; ++j) {
      const i64 w = n - (j + 1) * b;  // trailing width after panel j
      if (w > 0) {
        size_t d = tn_partial_doubles(m, b, (int)w, 0);
        if (d > pd) pd = d;
      }
      const i64 jb = (j + 1) * b;  // mCQR2GS re-orthogonalisation against jb columns
      if (variant == CQR_MCQR2GS && jb < n) {
        size_t d = tn_partial_doubles(m, (int)jb, b, 0);
        if (d > pd) pd = d;
      }
    }
  }
  if (halving && variant == CQR_MCQR2GS) {
    // every width of the chain b, h(b), h(h(b)), ..., 1 at every position it
    // can start from (a multiple of itself), after a panel of any wider width
    int chain[40], nc = 0;
    for (int w = b;; w = halved_width(w)) {
      chain[nc++] = w;
      if (w == 1) break;
    }
    for (int i = 0; i < nc; ++i) {
      const int w2 = chain[i];
      const size_t g = tn_partial_doubles(m, w2, w2, 1);
      if (g > pd) pd = g;
      for (i64 c0 = w2; c0 < n; c0 += w2) {
        for (int h = 0; h <= i; ++h) {
          const int w1 = chain[h];
          if (c0 >= w1 && c0 % w1 == 0) {
            const size_t d = tn_partial_doubles(m, w1, (int)(n - c0), 0);
            if (d > pd) pd = d;
          }
        }
        const size_t d = tn_partial_doubles(m, (int)c0, w2, 0);
        if (d > pd) pd = d;
      }
    }
  }
  L.part = take(sizeof(double) * pd);
  size_t oz = 0;
  if (emulated && variant == CQR_MCQR2GS) {  // Gram matrices; products with Y (b x w) and Z (jb x b) of Alg. 9
    oz = ozaki_workspace_bytes(m, b, b);
    for (int c0 = kTrsmEmuB; c0 < b; c0 += kTrsmEmuB) {  // the triangular solves' coupling products
      const size_t d = ozaki_nn_workspace_bytes(m, b - c0 < kTrsmEmuB ? b - c0 : kTrsmEmuB, c0);
      if (d > oz) oz = d;
    }
    for (i64 j = 1; j * b < n; ++j) {
      const size_t d[4] = {ozaki_workspace_bytes(m, b, (int)(n - j * b)), ozaki_workspace_bytes(m, (int)(j * b), b),
                           ozaki_nn_workspace_bytes(m, (int)(n - j * b), b),
                           ozaki_nn_workspace_bytes(m, b, (int)(j * b))};
      for (size_t x : d)
        if (x > oz) oz = x;
    }
  }
  L.oz = take(oz);
  L.total = off;
  static_assert(kStatusOffset == 0, "status word first");
  return L;
}

struct Work {
  int* status;
  int* skip;  // second-pass decision of the runtime repetition choice; panel test of the adaptive width
  double *W, *S1, *S2, *rinv, *Z, *R1, *R2, *part;
  void* oz;   // emulated projections and updates (null: native FP64)
};

Work bind(void* ws, const Layout& L) {
  char* p = (char*)ws;
  Work w;
  w.status = (int*)(p + L.status);
  w.skip = (int*)(p + L.skip);
  w.W = (double*)(p + L.W);
  w.S1 = (double*)(p + L.S1);
  w.S2 = (double*)(p + L.S2);
  w.rinv = (double*)(p + L.rinv);
  w.Z = (double*)(p + L.Z);
  w.R1 = (double*)(p + L.R1);
  w.R2 = (double*)(p + L.R2);
  w.part = (double*)(p + L.part);
  w.oz = nullptr;
  return w;
}

#define TRY(x)                            \
  do {                                    \
    cudaError_t e_ = (x);                 \
    if (e_ != cudaSuccess) return e_;     \
  } while (0)

// X := X U^{-1} for any width: kTrsmMaxB-column blocks, the coupling between
// blocks applied as an FMA update in ascending column order (so each element
// sees the same operation sequence as plain substitution).  With `oz` (the
// emulated variant) the coupling X_2 -= X_1 U_12 is one of the m-row
// products and runs on the tensor cores like the others; the substitutions
// within a block stay FP64.
cudaError_t trsm_any(i64 m, int b, double* X, i64 ldx, const double* U, i64 ldu, const double* rinv,
                     const int* status, cudaStream_t st, const int* skip = nullptr, void* oz = nullptr) {
  const int blk = oz ? kTrsmEmuB : kTrsmMaxB;
  for (int c0 = 0; c0 < b; c0 += blk) {
    const int cb = b - c0 < blk ? b - c0 : blk;
    if (c0 > 0 && oz)
      TRY(nn_update_emulated(m, cb, c0, X, ldx, U + (i64)c0 * ldu, ldu, X + (i64)c0 * ldx, ldx, oz, status, st));
    else if (c0 > 0)
      TRY(nn_product(m, cb, c0, X, ldx, U + (i64)c0 * ldu, ldu, X + (i64)c0 * ldx, ldx, -1.0, 1, 0, 0, status, st));
    TRY(trsm_rows(m, cb, X + (i64)c0 * ldx, ldx, U + c0 + (i64)c0 * ldu, ldu, rinv + c0, status, st, skip));
  }
  return cudaSuccess;
}

// X := X U^{-T} for any width (adjoint), blocks from the right.
cudaError_t trsm_t_any(i64 m, int b, double* X, i64 ldx, const double* U, i64 ldu, const double* rinv,
                       cudaStream_t st) {
  const int nblk = (b + kTrsmMaxB - 1) / kTrsmMaxB;
  for (int q = nblk - 1; q >= 0; --q) {
    const int c0 = q * kTrsmMaxB;
    const int cb = b - c0 < kTrsmMaxB ? b - c0 : kTrsmMaxB;
    const int c1 = c0 + cb;
    if (c1 < b)  // X[:, c0:c1] -= X[:, c1:b] * (U[c0:c1, c1:b])^T
      TRY(nn_product_t(m, cb, b - c1, X + (i64)c1 * ldx, ldx, U + c0 + (i64)c1 * ldu, ldu, 1, X + (i64)c0 * ldx,
                       ldx, -1.0, 1, 0, 0, nullptr, st));
    TRY(trsm_rows_transposed(m, cb, X + (i64)c0 * ldx, ldx, U + c0 + (i64)c0 * ldu, ldu, rinv + c0, st));
  }
  return cudaSuccess;
}

// Alg. 1 on the m x b panel X (in place): W = X^T X; W = U^T U; X := X U^{-1}.
// `second_pass_rule`: the runtime repetition choice (Sec. 7) for a second
// CholeskyQR pass -- U within 8u of I becomes I and the solve is skipped.
cudaError_t cqr_panel(i64 m, int b, double* X, i64 ldx, double* U, i64 ldu, const Work& w, int col0, int shift,
                      cudaStream_t st, bool second_pass_rule = false) {
  int* skip = second_pass_rule ? w.skip : nullptr;
  if (w.oz)  // emulated variant: the Gram W = X^T X on the tensor cores too (exactly symmetric)
    TRY(tn_product_emulated(m, b, b, X, ldx, X, ldx, w.oz, w.W, b, w.status, st));
  else
    TRY(tn_product(m, b, b, X, ldx, X, ldx, 1, w.part, w.W, b, w.status, st));
  TRY(chol_factor(b, w.W, b, U, ldu, w.rinv, col0, w.status, shift, m, st, skip));
  TRY(trsm_any(m, b, X, ldx, U, ldu, w.rinv, w.status, st, skip, w.oz));
  return cudaSuccess;
}

// Look-ahead (the overlap of the trailing update with the next panel's
// CholeskyQR that Sec. 7 lists as future work).  When a side stream is
// given, the update of step j is split: the next panel's b columns are
// updated first on the caller's stream, so its CQR (and, in Alg. 9, its
// re-orthogonalisation) starts at once, while the rest of the trailing
// update runs concurrently on the side stream; the next projection waits
// for it.  Each element still receives the same FMA sequence, so the
// results are bitwise those of the unsplit schedule; the overlap fills the
// GPU during the serial Cholesky islands, reductions and launch gaps.
struct Side {
  cudaStream_t s;
  cudaEvent_t to_side, to_main;
};

// A_{j:k} -= Qp Y with the split above.  Y is b x wd with leading dim ldy.
cudaError_t split_update(i64 m, int b, i64 wd, const double* Qp, i64 ldq, const double* Y, i64 ldy, double* Aj,
                         i64 lda, const int* status, cudaStream_t st, const Side* side, bool* pending) {
  if (side && wd > b) {
    TRY(cudaEventRecord(side->to_side, st));
    TRY(cudaStreamWaitEvent(side->s, side->to_side, 0));
    TRY(nn_product(m, (int)(wd - b), b, Qp, ldq, Y + (i64)b * ldy, ldy, Aj + (i64)b * lda, lda, -1.0, 1, 0, 0,
                   status, side->s));
    TRY(cudaEventRecord(side->to_main, side->s));
    *pending = true;
    return nn_product(m, b, b, Qp, ldq, Y, ldy, Aj, lda, -1.0, 1, 0, 0, status, st);
  }
  return nn_product(m, (int)wd, b, Qp, ldq, Y, ldy, Aj, lda, -1.0, 1, 0, 0, status, st);
}

cudaError_t join_side(cudaStream_t st, const Side* side, bool* pending) {
  if (side && *pending) {
    *pending = false;
    return cudaStreamWaitEvent(st, side->to_main, 0);
  }
  return cudaSuccess;
}

// Alg. 6 on X (m x n, in place), panels of width b; R (ldr) pre-zeroed.
cudaError_t cqrgs_run(i64 m, i64 n, int b, double* X, i64 ldx, double* R, i64 ldr, const Work& w, cudaStream_t st,
                      const Side* side) {
  const i64 k = n / b;
  bool pending = false;
  for (i64 j = 0; j < k; ++j) {
    const i64 jb = j * b;
    double* Xj = X + jb * ldx;
    {
      TracePhase ph("cqr", (int)j);
      TRY(cqr_panel(m, b, Xj, ldx, R + jb + jb * ldr, ldr, w, (int)jb, 0, st));
    }
    const i64 wd = n - jb - b;
    if (wd > 0) {
      TracePhase ph("project_update", (int)j);
      TRY(join_side(st, side, &pending));  // the rest of the previous update
      double* Yp = R + jb + (jb + b) * ldr;  // Y lands in R_{j,j+1:k}
      TRY(tn_product(m, b, (int)wd, Xj, ldx, Xj + (i64)b * ldx, ldx, 0, w.part, Yp, ldr, w.status, st));
      TRY(split_update(m, b, wd, Xj, ldx, Yp, ldr, Xj + (i64)b * ldx, ldx, w.status, st, side, &pending));
    }
  }
  return join_side(st, side, &pending);
}

// Host-buffer factorisation (cqr_factor_host): the copy stream that brings
// A's columns after the first panel in and takes every finished Q panel out.
struct HostIO {
  cudaStream_t cs;
  cudaEvent_t fork, in_done, panel_done, join;
  double* Qh;  // host destination of Q
  i64 ldqh;
  bool rest_pending;  // the main stream has not yet waited for in_done
};

// Columns [c0, c0 + w) of an m-row column-major matrix between two buffers
// (one copy; a 1-D copy when both are packed).
cudaError_t copy_cols(double* dst, i64 ldd, const double* src, i64 lds, i64 m, i64 c0, i64 w, cudaMemcpyKind kind,
                      cudaStream_t s) {
  if (w <= 0) return cudaSuccess;
  if (ldd == m && lds == m)
    return cudaMemcpyAsync(dst + c0 * ldd, src + c0 * lds, sizeof(double) * m * w, kind, s);
  return cudaMemcpy2DAsync(dst + c0 * ldd, sizeof(double) * ldd, src + c0 * lds, sizeof(double) * lds,
                           sizeof(double) * m, w, kind, s);
}

// Before the first m-row product that reads columns past the first panel.
cudaError_t io_wait_rest(HostIO* io, cudaStream_t st) {
  if (!io || !io->rest_pending) return cudaSuccess;
  io->rest_pending = false;
  return cudaStreamWaitEvent(st, io->in_done, 0);
}

// Q's columns [c0, c0 + w) are final (Alg. 9 step 1 / step 8) and no later
// kernel writes them: copy them out behind the work enqueued so far.
cudaError_t io_panel_out(HostIO* io, i64 m, const double* Q, i64 ldq, i64 c0, i64 w, cudaStream_t st) {
  if (!io) return cudaSuccess;
  TRY(cudaEventRecord(io->panel_done, st));
  TRY(cudaStreamWaitEvent(io->cs, io->panel_done, 0));
  return copy_cols(io->Qh, io->ldqh, Q, ldq, m, c0, w, cudaMemcpyDeviceToHost, io->cs);
}

// Alg. 9 on Q (m x n, in place); R (ldr) pre-zeroed.
cudaError_t mcqr2gs_run(i64 m, i64 n, int b, double* Q, i64 ldq, double* R, i64 ldr, const Work& w, cudaStream_t st,
                        const Side* side, bool adaptive, HostIO* io = nullptr) {
  const i64 k = n / b;
  bool pending = false;
  {  // step 1: [Q_1, R_11] = CQR2(A_1)
    TracePhase ph("cqr2_first_panel", 0);
    TRY(cqr_panel(m, b, Q, ldq, w.S1, b, w, 0, 0, st));
    TRY(cqr_panel(m, b, Q, ldq, w.S2, b, w, 0, 0, st, adaptive));
    TRY(nn_product(b, b, b, w.S2, b, w.S1, b, R, ldr, 1.0, 0, 1, 1, w.status, st));
    TRY(io_panel_out(io, m, Q, ldq, 0, b, st));
  }
  for (i64 j = 1; j < k; ++j) {
    const i64 jb = j * b, wd = n - jb;
    const double* Qprev = Q + (jb - b) * ldq;
    double* Aj = Q + jb * ldq;
    double* Yp = R + (jb - b) + jb * ldr;
    const int pj = (int)j;
    {  // steps 3-5: Y = Q_{j-1}^T A_{j:k}; A_{j:k} -= Q_{j-1} Y; R_{j-1,j:k} = Y
      TracePhase ph("project_update", pj);
      TRY(join_side(st, side, &pending));
      TRY(io_wait_rest(io, st));
      if (w.oz)
        TRY(tn_product_emulated(m, b, (int)wd, Qprev, ldq, Aj, ldq, w.oz, Yp, ldr, w.status, st));
      else
        TRY(tn_product(m, b, (int)wd, Qprev, ldq, Aj, ldq, 0, w.part, Yp, ldr, w.status, st));
      if (w.oz)  // the emulated update uses w.oz, so it stays on this stream (no look-ahead split)
        TRY(nn_update_emulated(m, (int)wd, b, Qprev, ldq, Yp, ldr, Aj, ldq, w.oz, w.status, st));
      else
        TRY(split_update(m, b, wd, Qprev, ldq, Yp, ldr, Aj, ldq, w.status, st, side, &pending));
    }
    {  // step 6: [P, S1] = CQR(A_j)
      TracePhase ph("cqr", pj);
      TRY(cqr_panel(m, b, Aj, ldq, w.S1, b, w, (int)jb, 0, st));
    }
    {  // step 7: Z = Q_{1:j-1}^T P; P -= Q_{1:j-1} Z
      TracePhase ph("reorthogonalise", pj);
      if (w.oz)
        TRY(tn_product_emulated(m, (int)jb, b, Q, ldq, Aj, ldq, w.oz, w.Z, jb, w.status, st));
      else
        TRY(tn_product(m, (int)jb, b, Q, ldq, Aj, ldq, 0, w.part, w.Z, jb, w.status, st));
      if (w.oz)
        TRY(nn_update_emulated(m, b, (int)jb, Q, ldq, w.Z, jb, Aj, ldq, w.oz, w.status, st));
      else
        TRY(nn_product(m, b, (int)jb, Q, ldq, w.Z, jb, Aj, ldq, -1.0, 1, 0, 0, w.status, st));
    }
    {  // step 8: [Q_j, S2] = CQR(P)
      TracePhase ph("cqr_final", pj);
      TRY(cqr_panel(m, b, Aj, ldq, w.S2, b, w, (int)jb, 0, st, adaptive));
      TRY(io_panel_out(io, m, Q, ldq, jb, b, st));
    }
    {  // R_jj = S2 S1;  R_{1:j-1,j} += Z S1
      TracePhase ph("r_update", pj);
      TRY(nn_product(b, b, b, w.S2, b, w.S1, b, R + jb + jb * ldr, ldr, 1.0, 0, 1, 1, w.status, st));
      TRY(nn_product(jb, b, b, w.Z, jb, w.S1, b, R + jb * ldr, ldr, 1.0, 1, 0, 1, w.status, st));
    }
  }
  return join_side(st, side, &pending);
}

// Alg. 9 with the adaptive panel width (CQR_HALVE): the first CholeskyQR of
// every panel (step 1's first pass, step 6) is tested on the device (the
// Cholesky kernel's panel test) and the host reads the decision before it
// enqueues the triangular solve; a rejected panel, left untouched, is
// retried with halved_width(b), which every later panel keeps.  The same
// rule as the oracle's or_mcqr2gs_halving; one host synchronisation per
// attempt.  *b_final receives the last panel's width.
cudaError_t mcqr2gs_halving_run(i64 m, i64 n, int b, double* Q, i64 ldq, double* R, i64 ldr, const Work& w,
                                cudaStream_t st, bool adaptive, int* b_final, HostIO* io = nullptr) {
  int bw = b, bprev = 0;
  for (i64 c0 = 0; c0 < n;) {
    double* Aj = Q + c0 * ldq;
    const int pc = (int)c0;
    if (c0 > 0) {  // steps 3-5 with the previous panel (its own width)
      TracePhase ph("project_update", pc);
      TRY(io_wait_rest(io, st));
      const double* Qprev = Q + (c0 - bprev) * ldq;
      double* Yp = R + (c0 - bprev) + c0 * ldr;
      TRY(tn_product(m, bprev, (int)(n - c0), Qprev, ldq, Aj, ldq, 0, w.part, Yp, ldr, w.status, st));
      TRY(nn_product(m, (int)(n - c0), bprev, Qprev, ldq, Yp, ldr, Aj, ldq, -1.0, 1, 0, 0, w.status, st));
    }
    for (;;) {  // the first CholeskyQR's Gram and Cholesky, with the panel test
      TracePhase ph("panel_test", pc);
      int rej = 0;
      TRY(cudaMemsetAsync(w.skip, 0, sizeof(int), st));
      TRY(tn_product(m, bw, bw, Aj, ldq, Aj, ldq, 1, w.part, w.W, bw, w.status, st));
      TRY(chol_factor(bw, w.W, bw, w.S1, bw, w.rinv, (int)c0, w.status, 0, m, st, nullptr, w.skip));
      TRY(cudaMemcpyAsync(&rej, w.skip, sizeof(int), cudaMemcpyDeviceToHost, st));
      TRY(cudaStreamSynchronize(st));
      if (!rej) break;
      bw = halved_width(bw);
    }
    {
      TracePhase ph(c0 > 0 ? "cqr" : "cqr2_first_panel", pc);
      TRY(trsm_any(m, bw, Aj, ldq, w.S1, bw, w.rinv, w.status, st));
    }
    if (c0 > 0) {  // step 7
      TracePhase ph("reorthogonalise", pc);
      TRY(tn_product(m, (int)c0, bw, Q, ldq, Aj, ldq, 0, w.part, w.Z, c0, w.status, st));
      TRY(nn_product(m, bw, (int)c0, Q, ldq, w.Z, c0, Aj, ldq, -1.0, 1, 0, 0, w.status, st));
    }
    {  // step 1's second pass / step 8
      TracePhase ph(c0 > 0 ? "cqr_final" : "cqr2_first_panel", pc);
      TRY(cqr_panel(m, bw, Aj, ldq, w.S2, bw, w, (int)c0, 0, st, adaptive));
      TRY(io_panel_out(io, m, Q, ldq, c0, bw, st));
    }
    {  // R_jj = S2 S1;  R_{1:j-1,j} += Z S1
      TracePhase ph("r_update", pc);
      TRY(nn_product(bw, bw, bw, w.S2, bw, w.S1, bw, R + c0 + c0 * ldr, ldr, 1.0, 0, 1, 1, w.status, st));
      if (c0 > 0) TRY(nn_product(c0, bw, bw, w.Z, c0, w.S1, bw, R + c0 * ldr, ldr, 1.0, 1, 0, 1, w.status, st));
    }
    bprev = bw;
    c0 += bw;
  }
  *b_final = bw;
  return cudaSuccess;
}

cudaError_t factor_run(i64 m, i64 n, int b, double* Q, i64 ldq, double* R, i64 ldr, int variant, const Work& w,
                       cudaStream_t st, const Side* side = nullptr, bool adaptive = false, HostIO* io = nullptr) {
  switch (variant) {
    case CQR_MCQR2GS:
      return mcqr2gs_run(m, n, b, Q, ldq, R, ldr, w, st, side, adaptive, io);
    case CQR_CQR2GS: {
      TRY(cudaMemsetAsync(w.R1, 0, sizeof(double) * n * n, st));
      TRY(cudaMemsetAsync(w.R2, 0, sizeof(double) * n * n, st));
      {
        TracePhase ph("cqrgs_pass", 0);
        TRY(cqrgs_run(m, n, b, Q, ldq, w.R1, n, w, st, side));
      }
      {
        TracePhase ph("cqrgs_pass", 1);
        TRY(cqrgs_run(m, n, b, Q, ldq, w.R2, n, w, st, side));
      }
      TracePhase ph("r_update", -1);
      return nn_product(n, (int)n, (int)n, w.R2, n, w.R1, n, R, ldr, 1.0, 0, 1, 1, w.status, st);
    }
    case CQR_CQR2: {
      TracePhase ph("cqr2", -1);
      TRY(cqr_panel(m, (int)n, Q, ldq, w.S1, n, w, 0, 0, st));
      TRY(cqr_panel(m, (int)n, Q, ldq, w.S2, n, w, 0, 0, st));
      return nn_product(n, (int)n, (int)n, w.S2, n, w.S1, n, R, ldr, 1.0, 0, 1, 1, w.status, st);
    }
    case CQR_SCQR3: {
      TracePhase ph("scqr3", -1);
      TRY(cqr_panel(m, (int)n, Q, ldq, w.R1, n, w, 0, 1, st));  // Alg. 5 step 1: sCQR
      TRY(cqr_panel(m, (int)n, Q, ldq, w.S1, n, w, 0, 0, st));  // step 2: CQR2
      TRY(cqr_panel(m, (int)n, Q, ldq, w.S2, n, w, 0, 0, st));
      TRY(nn_product(n, (int)n, (int)n, w.S2, n, w.S1, n, w.R2, n, 1.0, 0, 1, 1, w.status, st));
      return nn_product(n, (int)n, (int)n, w.R2, n, w.R1, n, R, ldr, 1.0, 0, 1, 1, w.status, st);
    }
    default:
      return cudaErrorInvalidValue;
  }
}

// Per-device side stream for the look-ahead of single factorisations.  The
// enqueue of one factorisation holds the mutex, so concurrent host threads
// do not interleave their event records.
std::mutex g_side_mu;
Side g_side[64];
bool g_side_ok[64] = {};

const Side* get_side() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!g_side_ok[dev]) {
    Side& s = g_side[dev];
    if (cudaStreamCreateWithFlags(&s.s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&s.to_side, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&s.to_main, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    g_side_ok[dev] = true;
  }
  return &g_side[dev];
}

// Per-device copy stream and events of cqr_factor_host; the enqueue of one
// call holds the mutex (the events are shared).
std::mutex g_io_mu;
HostIO g_io[64];
bool g_io_ok[64] = {};

HostIO* get_io() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!g_io_ok[dev]) {
    HostIO& h = g_io[dev];
    if (cudaStreamCreateWithFlags(&h.cs, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    for (cudaEvent_t* e : {&h.fork, &h.in_done, &h.panel_done, &h.join})
      if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    g_io_ok[dev] = true;
  }
  return &g_io[dev];
}

// Caller-registered allocator for calls made with workspace == NULL.
struct Allocator {
  cqr_alloc_fn alloc = nullptr;
  cqr_free_fn free = nullptr;
  void* ctx = nullptr;
};
std::mutex g_alloc_mu;
Allocator g_alloc;

bool registered_allocator(Allocator* out) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  *out = g_alloc;
  return out->alloc != nullptr;
}

// workspace == NULL: take `bytes` from the registered allocator, run `body`
// on it, synchronise `st`, read the status word at offset 0 when asked, and
// hand the memory back.  Returns body's nonzero code, CQR_ERR_ALLOC, a CUDA
// error, or the status word (0 when not read).
template <class F>
int with_allocated_workspace(const Allocator& al, size_t bytes, cudaStream_t st, bool read_status, F&& body) {
  void* ws = al.alloc(bytes, (cqr_stream_t)st, al.ctx);
  if (!ws) return CQR_ERR_ALLOC;
  if ((uintptr_t)ws & 255) {
    al.free(ws, bytes, (cqr_stream_t)st, al.ctx);
    return CQR_ERR_ALLOC;
  }
  int rc = body(ws);
  int status = 0;
  if (rc == 0 && read_status) {
    if (cudaMemcpyAsync(&status, ws, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = CQR_ERR_CUDA;
  }
  // the memory goes back only once the stream has finished with it
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == 0) rc = CQR_ERR_CUDA;
  al.free(ws, bytes, (cqr_stream_t)st, al.ctx);
  return rc != 0 ? rc : status;
}

bool overlaps(const double* a, i64 lda, i64 m, i64 n, const double* b, i64 ldb) {
  const char* a0 = (const char*)a;
  const char* a1 = (const char*)(a + (n - 1) * lda + m);
  const char* b0 = (const char*)b;
  const char* b1 = (const char*)(b + (n - 1) * ldb + m);
  return a0 < b1 && b0 < a1;
}

}  // namespace

extern "C" {

int cqr_set_allocator(cqr_alloc_fn alloc, cqr_free_fn free_fn, void* ctx) {
  if (!alloc && free_fn) return -1;
  if (alloc && !free_fn) return -2;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.free = free_fn;
  g_alloc.ctx = ctx;
  return 0;
}

int cqr_default_panel(int64_t n) {
  if (n <= 0) return 0;
  i64 cap = (n + 2) / 3;
  if (cap > 256) cap = 256;
  if (cap < 1) cap = 1;
  for (i64 b = cap; b >= 1; --b)
    if (n % b == 0) return (int)b;
  return 1;
}

static int resolve_panel(int64_t n, int panel_b, int variant) {
  if (variant == CQR_CQR2 || variant == CQR_SCQR3) return (int)n;
  return panel_b == 0 ? cqr_default_panel(n) : panel_b;
}

size_t cqr_workspace_size(int64_t m, int64_t n, int panel_b, int variant_flags) {
  const bool emulated = (variant_flags & CQR_EMULATED) != 0;
  const bool halving = (variant_flags & CQR_HALVE) != 0;
  const int variant = variant_flags & ~(CQR_LOOKAHEAD | CQR_ADAPTIVE | CQR_EMULATED | CQR_HALVE);
  if (m < 1 || n < 1 || m < n || variant < 0 || variant > 3) return 0;
  if ((variant == CQR_CQR2 || variant == CQR_SCQR3) && n > CQR_MAX_PANEL) return 0;
  const int b = resolve_panel(n, panel_b, variant);
  if (b < 1 || b > CQR_MAX_PANEL || n % b) return 0;
  if ((emulated || halving) && variant != CQR_MCQR2GS) return 0;
  return make_layout(m, n, b, variant, emulated, halving).total;
}

int cqr_factor(int64_t m, int64_t n, double* A, int64_t lda, int panel_b, double* Q, int64_t ldq, double* R,
               int64_t ldr, int variant_flags, void* workspace, size_t ws_bytes, cqr_stream_t stream) {
  const bool lookahead = (variant_flags & CQR_LOOKAHEAD) != 0;
  const bool adaptive = (variant_flags & CQR_ADAPTIVE) != 0;
  const bool emulated = (variant_flags & CQR_EMULATED) != 0;
  const bool halving = (variant_flags & CQR_HALVE) != 0;
  const int variant = variant_flags & ~(CQR_LOOKAHEAD | CQR_ADAPTIVE | CQR_EMULATED | CQR_HALVE);
  if (m < 1 || m < n) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (variant < 0 || variant > 3) return -10;
  if ((variant == CQR_CQR2 || variant == CQR_SCQR3) && n > CQR_MAX_PANEL) return -2;  // one panel, b = n
  const int b = resolve_panel(n, panel_b, variant);
  if (panel_b < 0 || b < 1 || b > CQR_MAX_PANEL || n % b) return -5;
  if (!Q) return -6;
  if (ldq < m || (Q == A && ldq != lda)) return -7;
  if (Q != A && overlaps(A, lda, m, n, Q, ldq)) return -6;
  if (!R) return -8;
  if (ldr < n) return -9;
  if ((emulated || adaptive || halving) && variant != CQR_MCQR2GS) return -10;
  if (halving && (emulated || lookahead)) return -10;
  const Layout L = make_layout(m, n, b, variant, emulated, halving);
  cudaStream_t st = (cudaStream_t)stream;
  if (!workspace) {
    Allocator al;
    if (!registered_allocator(&al)) return -11;
    return with_allocated_workspace(al, L.total, st, true, [&](void* ws) {
      return cqr_factor(m, n, A, lda, panel_b, Q, ldq, R, ldr, variant_flags, ws, L.total, stream);
    });
  }
  if ((uintptr_t)workspace & 255) return -11;
  if (ws_bytes < L.total) return -12;
  Work w = bind(workspace, L);
  if (emulated) w.oz = (char*)workspace + L.oz;
  cudaGetLastError();  // clear stale errors from earlier, unrelated calls
  if (cudaMemsetAsync(w.status, 0, sizeof(int), st) != cudaSuccess) return CQR_ERR_CUDA;
  if (Q != A && cudaMemcpy2DAsync(Q, sizeof(double) * ldq, A, sizeof(double) * lda, sizeof(double) * m, n,
                                  cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return CQR_ERR_CUDA;
  if (cudaMemset2DAsync(R, sizeof(double) * ldr, 0, sizeof(double) * n, n, st) != cudaSuccess) return CQR_ERR_CUDA;
  if (halving) {
    int b_final = b;
    if (mcqr2gs_halving_run(m, n, b, Q, ldq, R, ldr, w, st, adaptive, &b_final) != cudaSuccess) return CQR_ERR_CUDA;
    if (cudaMemcpyAsync((char*)workspace + kPanelOffset, &b_final, sizeof(int), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return CQR_ERR_CUDA;
  } else if (lookahead && (variant == CQR_MCQR2GS || variant == CQR_CQR2GS)) {
    std::lock_guard<std::mutex> lk(g_side_mu);
    const Side* side = get_side();
    if (!side) return CQR_ERR_CUDA;
    if (factor_run(m, n, b, Q, ldq, R, ldr, variant, w, st, side, adaptive) != cudaSuccess) return CQR_ERR_CUDA;
  } else if (factor_run(m, n, b, Q, ldq, R, ldr, variant, w, st, nullptr, adaptive) != cudaSuccess) {
    return CQR_ERR_CUDA;
  }
  return 0;
}

int cqr_factor_host(int64_t m, int64_t n, const double* A, int64_t lda, int panel_b, double* Q, int64_t ldq,
                    double* R, int64_t ldr, int variant_flags, double* Qd, int64_t ldqd, double* Rd, int64_t ldrd,
                    void* workspace, size_t ws_bytes, cqr_stream_t stream) {
  const bool lookahead = (variant_flags & CQR_LOOKAHEAD) != 0;
  const bool adaptive = (variant_flags & CQR_ADAPTIVE) != 0;
  const bool emulated = (variant_flags & CQR_EMULATED) != 0;
  const bool halving = (variant_flags & CQR_HALVE) != 0;
  const int variant = variant_flags & ~(CQR_LOOKAHEAD | CQR_ADAPTIVE | CQR_EMULATED | CQR_HALVE);
  if (m < 1 || m < n) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (variant < 0 || variant > 3) return -10;
  if ((variant == CQR_CQR2 || variant == CQR_SCQR3) && n > CQR_MAX_PANEL) return -2;
  const int b = resolve_panel(n, panel_b, variant);
  if (panel_b < 0 || b < 1 || b > CQR_MAX_PANEL || n % b) return -5;
  if (!Q) return -6;
  if (ldq < m || ((const double*)Q == A && ldq != lda)) return -7;
  if ((const double*)Q != A && overlaps(A, lda, m, n, Q, ldq)) return -6;
  if (!R) return -8;
  if (ldr < n) return -9;
  if ((emulated || adaptive || halving) && variant != CQR_MCQR2GS) return -10;
  if (halving && (emulated || lookahead)) return -10;
  if (!Qd) return -13;
  if (ldqd < m) return -14;
  if (!Rd) return -15;
  if (ldrd < n) return -16;
  {  // Rd's extent (n x n, ldrd) against Qd's (m x n, ldqd)
    const char *q0 = (const char*)Qd, *q1 = (const char*)(Qd + (n - 1) * ldqd + m);
    const char *r0 = (const char*)Rd, *r1 = (const char*)(Rd + (n - 1) * ldrd + n);
    if (q0 < r1 && r0 < q1) return -15;
  }
  const Layout L = make_layout(m, n, b, variant, emulated, halving);
  cudaStream_t st = (cudaStream_t)stream;
  if (!workspace) {
    Allocator al;
    if (!registered_allocator(&al)) return -11;
    return with_allocated_workspace(al, L.total, st, true, [&](void* ws) {
      return cqr_factor_host(m, n, A, lda, panel_b, Q, ldq, R, ldr, variant_flags, Qd, ldqd, Rd, ldrd, ws, L.total,
                             stream);
    });
  }
  if ((uintptr_t)workspace & 255) return -11;
  if (ws_bytes < L.total) return -12;
  Work w = bind(workspace, L);
  if (emulated) w.oz = (char*)workspace + L.oz;
  cudaGetLastError();
  std::lock_guard<std::mutex> lk(g_io_mu);
  HostIO* io = get_io();
  if (!io) return CQR_ERR_CUDA;
  io->Qh = Q;
  io->ldqh = ldq;
  io->rest_pending = false;
  // Alg. 9 overlaps; the other variants copy in, factor and copy out
  const bool overlap = variant == CQR_MCQR2GS;
  const i64 first = overlap ? b : n;
  if (cudaMemsetAsync(w.status, 0, sizeof(int), st) != cudaSuccess) return CQR_ERR_CUDA;
  if (cudaMemset2DAsync(Rd, sizeof(double) * ldrd, 0, sizeof(double) * n, n, st) != cudaSuccess) return CQR_ERR_CUDA;
  if (copy_cols(Qd, ldqd, A, lda, m, 0, first, cudaMemcpyHostToDevice, st) != cudaSuccess) return CQR_ERR_CUDA;
  // the copy stream starts behind the first panel's copy (which it does not
  // share the link with) and everything the caller enqueued before
  if (cudaEventRecord(io->fork, st) != cudaSuccess || cudaStreamWaitEvent(io->cs, io->fork, 0) != cudaSuccess)
    return CQR_ERR_CUDA;
  // From here on an error still joins the copy stream into `stream`, so that
  // no copy of the caller's host buffers outlives the call's stream work.
  auto fail = [&]() {
    if (cudaEventRecord(io->join, io->cs) == cudaSuccess) cudaStreamWaitEvent(st, io->join, 0);
    return CQR_ERR_CUDA;
  };
  if (first < n) {
    if (copy_cols(Qd, ldqd, A, lda, m, first, n - first, cudaMemcpyHostToDevice, io->cs) != cudaSuccess ||
        cudaEventRecord(io->in_done, io->cs) != cudaSuccess)
      return fail();
    io->rest_pending = true;
  }
  HostIO* pio = overlap ? io : nullptr;
  int b_final = b;
  cudaError_t e;
  if (halving) {
    e = mcqr2gs_halving_run(m, n, b, Qd, ldqd, Rd, ldrd, w, st, adaptive, &b_final, pio);
  } else if (lookahead && (variant == CQR_MCQR2GS || variant == CQR_CQR2GS)) {
    std::lock_guard<std::mutex> lk2(g_side_mu);
    const Side* side = get_side();
    e = side ? factor_run(m, n, b, Qd, ldqd, Rd, ldrd, variant, w, st, side, adaptive, pio) : cudaErrorUnknown;
  } else {
    e = factor_run(m, n, b, Qd, ldqd, Rd, ldrd, variant, w, st, nullptr, adaptive, pio);
  }
  if (e != cudaSuccess) return fail();
  if (io_wait_rest(io, st) != cudaSuccess) return fail();  // n == b: nothing waited for it
  if (!overlap && copy_cols(Q, ldq, Qd, ldqd, m, 0, n, cudaMemcpyDeviceToHost, st) != cudaSuccess) return fail();
  // join the copy stream, then R
  if (cudaEventRecord(io->join, io->cs) != cudaSuccess || cudaStreamWaitEvent(st, io->join, 0) != cudaSuccess)
    return CQR_ERR_CUDA;
  if (copy_cols(R, ldr, Rd, ldrd, n, 0, n, cudaMemcpyDeviceToHost, st) != cudaSuccess) return CQR_ERR_CUDA;
  if (halving) {
    if (cudaMemcpyAsync((char*)workspace + kPanelOffset, &b_final, sizeof(int), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return CQR_ERR_CUDA;
  }
  return 0;
}

int cqr_read_panel_width(const void* workspace, cqr_stream_t stream, int* panel_b) {
  if (!workspace || !panel_b) return -1;
  int h = 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&h, (const char*)workspace + kPanelOffset, sizeof(int), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return CQR_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CQR_ERR_CUDA;
  *panel_b = h;
  return 0;
}

int cqr_batched_panel_widths(int batch, const void* workspace, cqr_stream_t stream, int* panel_b) {
  if (batch < 1) return -1;
  if (!workspace) return -2;
  if (!panel_b) return -4;
  return batched_persistent_panels(batch, workspace, panel_b, (cudaStream_t)stream) == cudaSuccess ? 0
                                                                                                  : CQR_ERR_CUDA;
}

int cqr_read_status(const void* workspace, cqr_stream_t stream, int* status) {
  if (!workspace || !status) return -1;
  int h = 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&h, workspace, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CQR_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CQR_ERR_CUDA;
  *status = h;
  return 0;
}

size_t cqr_backward_workspace_size(int64_t m, int64_t n) {
  if (m < 1 || n < 1 || m < n) return 0;
  size_t off = 0;
  off = align256(off + sizeof(double) * n * n);  // G
  off = align256(off + sizeof(double) * n * n);  // T
  off = align256(off + sizeof(double) * n * n);  // M
  off = align256(off + sizeof(double) * n);      // rinv
  off = align256(off + sizeof(double) * tn_partial_doubles(m, (int)n, (int)n, 0));
  return off;
}

int cqr_backward(int64_t m, int64_t n, const double* Q, int64_t ldq, const double* R, int64_t ldr,
                 const double* dQ, int64_t lddq, const double* dR, int64_t lddr, double* dA, int64_t ldda,
                 void* workspace, size_t ws_bytes, cqr_stream_t stream) {
  if (m < 1 || m < n) return -1;
  if (n < 1) return -2;
  if (!Q) return -3;
  if (ldq < m) return -4;
  if (!R) return -5;
  if (ldr < n) return -6;
  if (dQ && lddq < m) return -8;
  if (dR && lddr < n) return -10;
  if (!dA) return -11;
  if (ldda < m) return -12;
  if (overlaps(dA, ldda, m, n, Q, ldq) || (dQ && overlaps(dA, ldda, m, n, dQ, lddq))) return -11;
  cudaStream_t st = (cudaStream_t)stream;
  if (!workspace) {
    Allocator al;
    if (!registered_allocator(&al)) return -13;
    const size_t need = cqr_backward_workspace_size(m, n);
    return with_allocated_workspace(al, need, st, false, [&](void* ws) {
      return cqr_backward(m, n, Q, ldq, R, ldr, dQ, lddq, dR, lddr, dA, ldda, ws, need, stream);
    });
  }
  if ((uintptr_t)workspace & 255) return -13;
  if (ws_bytes < cqr_backward_workspace_size(m, n)) return -14;
  char* p = (char*)workspace;
  size_t off = 0;
  double* G = (double*)(p + off);
  off = align256(off + sizeof(double) * n * n);
  double* T = (double*)(p + off);
  off = align256(off + sizeof(double) * n * n);
  double* M = (double*)(p + off);
  off = align256(off + sizeof(double) * n * n);
  double* rinv = (double*)(p + off);
  off = align256(off + sizeof(double) * n);
  double* part = (double*)(p + off);
  TracePhase ph("backward", -1);
  cudaGetLastError();
  const int nn = (int)n;
  // G = Qbar^T Q
  if (dQ) {
    if (tn_product(m, nn, nn, dQ, lddq, Q, ldq, 0, part, G, n, nullptr, st) != cudaSuccess) return CQR_ERR_CUDA;
  } else if (cudaMemsetAsync(G, 0, sizeof(double) * n * n, st) != cudaSuccess) {
    return CQR_ERR_CUDA;
  }
  // T = R Rbar^T (R upper: k >= row)
  if (dR) {
    if (nn_product_t(n, nn, nn, R, ldr, dR, lddr, 1, T, n, 1.0, 0, 1, 0, nullptr, st) != cudaSuccess)
      return CQR_ERR_CUDA;
  } else if (cudaMemsetAsync(T, 0, sizeof(double) * n * n, st) != cudaSuccess) {
    return CQR_ERR_CUDA;
  }
  if (backward_middle(nn, T, G, M, st) != cudaSuccess) return CQR_ERR_CUDA;
  // B = Qbar + Q M  (into dA)
  if (dQ) {
    if (cudaMemcpy2DAsync(dA, sizeof(double) * ldda, dQ, sizeof(double) * lddq, sizeof(double) * m, n,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return CQR_ERR_CUDA;
  }
  if (nn_product(m, nn, nn, Q, ldq, M, n, dA, ldda, 1.0, dQ ? 1 : 0, 0, 0, nullptr, st) != cudaSuccess)
    return CQR_ERR_CUDA;
  // Abar = B R^{-T}
  if (diag_reciprocal(nn, R, ldr, rinv, st) != cudaSuccess) return CQR_ERR_CUDA;
  if (trsm_t_any(m, nn, dA, ldda, R, ldr, rinv, st) != cudaSuccess) return CQR_ERR_CUDA;
  return 0;
}

// ---------------------------------------------------------------------------
// Batched factorisation.  The matrices are spread over a pool of library-owned
// non-blocking streams (largest work first, each to the least-loaded stream);
// every stream owns one slice of the workspace.  The pool is forked from the
// caller's stream with an event and joined back into it, so the whole call is
// ordered on the caller's stream and can be captured into a CUDA graph.  Each
// matrix runs exactly the kernel sequence of a single cqr_factor() call with
// the same sizes and panel width, so its result is bitwise identical; the
// gain comes from running the small grids, the one-block Cholesky islands and
// the reductions of different matrices concurrently.
namespace {

constexpr int kBatchStreams = 16;

struct StreamPool {
  cudaStream_t s[kBatchStreams];
  cudaEvent_t done[kBatchStreams];
  cudaEvent_t fork;
  int device = -1;
  bool ok = false;
};
StreamPool g_pool[64];  // per device
// One batched call at a time enqueues on the pool: the fork event and the
// streams are shared, so two host threads interleaving their records would
// make one batch wait on the other's fork point.
std::mutex g_pool_mu;

StreamPool* get_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  StreamPool& p = g_pool[dev];
  if (!p.ok) {
    for (int i = 0; i < kBatchStreams; ++i) {
      if (cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
      if (cudaEventCreateWithFlags(&p.done[i], cudaEventDisableTiming) != cudaSuccess) return nullptr;
    }
    if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    p.device = dev;
    p.ok = true;
  }
  return &p;
}

size_t batched_slice(int batch, const int64_t* m, const int64_t* n, const int* panel_b, int variant) {
  size_t mx = 256;
  for (int i = 0; i < batch; ++i) {
    const size_t s = cqr_workspace_size(m[i], n[i], panel_b[i], variant);
    if (s == 0) return 0;
    if (s > mx) mx = s;
  }
  return align256(mx);
}

}  // namespace

namespace {

// Batched variant word: base variant | CQR_HALVE | CQR_BATCH_POOL | CQR_BATCH_GROUP(G).
struct BatchMode {
  int variant, G;
  bool halve, pool_forced;
};
BatchMode batch_mode(int flags) {
  BatchMode b;
  b.variant = flags & 0xFF;
  b.halve = (flags & CQR_HALVE) != 0;
  b.pool_forced = (flags & CQR_BATCH_POOL) != 0;
  b.G = (flags >> 16) & 0xFF;
  return b;
}
bool batch_flags_ok(int flags) {
  return (flags & ~(0xFF | CQR_HALVE | CQR_BATCH_POOL | 0xFF0000)) == 0;
}

// The persistent path takes mCQR2GS batches of matrices with n <= 128 and
// n, b multiples of 4, unless the stream pool is forced.
bool use_persistent(int batch, const int64_t* m, const int64_t* n, const int* panel_b, const BatchMode& md) {
  if (md.variant != CQR_MCQR2GS || md.pool_forced) return false;
  std::vector<int> b((size_t)batch);
  for (int i = 0; i < batch; ++i) b[i] = resolve_panel(n[i], panel_b[i], md.variant);
  return batched_persistent_eligible(batch, m, n, b.data());
}

}  // namespace

size_t cqr_batched_workspace_size(int batch, const int64_t* m, const int64_t* n, const int* panel_b, int flags) {
  const BatchMode md = batch_mode(flags);
  if (!batch_flags_ok(flags) || batch < 0 || (md.variant != CQR_MCQR2GS && md.variant != CQR_CQR2GS)) return 0;
  if (batch == 0) return 256;
  if (!m || !n || !panel_b) return 0;
  const int variant = md.variant;
  for (int i = 0; i < batch; ++i)
    if (cqr_workspace_size(m[i], n[i], panel_b[i], variant) == 0) return 0;
  if (use_persistent(batch, m, n, panel_b, md)) return batched_persistent_workspace(batch);
  if (md.halve) return 0;  // the adaptive width of a batch runs on the persistent path only
  const size_t slice = batched_slice(batch, m, n, panel_b, variant);
  if (slice == 0) return 0;
  const int ns = batch < kBatchStreams ? batch : kBatchStreams;
  return slice * (size_t)ns;
}

int cqr_factor_batched(int batch, const int64_t* m, const int64_t* n, const int64_t* lda, const int* panel_b,
                       double* const* A, double* const* Q, double* const* R, int flags, int* status,
                       void* workspace, size_t ws_bytes, cqr_stream_t stream) {
  const BatchMode md = batch_mode(flags);
  const int variant = md.variant;
  if (batch < 0) return -1;
  if (batch == 0) return 0;
  if (!m || !n || !lda || !panel_b) return -2;
  if (!A || !Q || !R) return -6;
  if (!batch_flags_ok(flags) || (variant != CQR_MCQR2GS && variant != CQR_CQR2GS)) return -9;
  if (!status) return -10;
  for (int i = 0; i < batch; ++i) {
    if (m[i] < 1 || n[i] < 1 || m[i] < n[i] || lda[i] < m[i]) return -2;
    const int b = resolve_panel(n[i], panel_b[i], variant);
    if (panel_b[i] < 0 || b < 1 || b > CQR_MAX_PANEL || n[i] % b) return -5;
    if (!A[i] || !Q[i] || !R[i]) return -6;
    if (Q[i] != A[i] && overlaps(A[i], lda[i], m[i], n[i], Q[i], lda[i])) return -7;
  }
  const bool persistent = use_persistent(batch, m, n, panel_b, md);
  if (md.halve && !persistent) return -9;
  if (!workspace) {
    Allocator al;
    if (!registered_allocator(&al)) return -11;
    const size_t need = cqr_batched_workspace_size(batch, m, n, panel_b, flags);
    return with_allocated_workspace(al, need, (cudaStream_t)stream, false, [&](void* ws) {
      return cqr_factor_batched(batch, m, n, lda, panel_b, A, Q, R, flags, status, ws, need, stream);
    });
  }
  if ((uintptr_t)workspace & 255) return -11;
  if (ws_bytes < cqr_batched_workspace_size(batch, m, n, panel_b, flags)) return -12;
  TracePhase ph("batched", batch);
  if (persistent) {
    const int grid = batched_persistent_grid();
    int G = md.G;
    if (G == 0)  // default: the largest divisor of the grid that is <= 8
      for (G = 8; grid % G; --G) {
      }
    if (grid % G) return -9;
    std::vector<int> b((size_t)batch);
    for (int i = 0; i < batch; ++i) b[i] = resolve_panel(n[i], panel_b[i], variant);
    cudaGetLastError();
    return batched_persistent_run(batch, m, n, lda, b.data(), A, Q, R, status, workspace, G, md.halve,
                                  (cudaStream_t)stream) == cudaSuccess
               ? 0
               : CQR_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  StreamPool* pool = get_pool();
  if (!pool) return CQR_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  cudaGetLastError();
  const size_t slice = batched_slice(batch, m, n, panel_b, variant);
  const int ns = batch < kBatchStreams ? batch : kBatchStreams;
  // largest work first, each to the least-loaded stream
  int* order = new int[batch];
  double* work = new double[batch];
  for (int i = 0; i < batch; ++i) {
    order[i] = i;
    work[i] = 4.0 * (double)m[i] * (double)n[i] * (double)n[i];
  }
  for (int i = 1; i < batch; ++i) {  // insertion sort by decreasing work (stable)
    int v = order[i], j = i - 1;
    while (j >= 0 && work[order[j]] < work[v]) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = v;
  }
  double load[kBatchStreams] = {0};
  int rc = 0;
  if (cudaMemsetAsync(status, 0, sizeof(int) * batch, st) != cudaSuccess || cudaEventRecord(pool->fork, st) != cudaSuccess)
    rc = CQR_ERR_CUDA;
  for (int k = 0; k < ns && rc == 0; ++k)
    if (cudaStreamWaitEvent(pool->s[k], pool->fork, 0) != cudaSuccess) rc = CQR_ERR_CUDA;
  for (int q = 0; q < batch && rc == 0; ++q) {
    const int i = order[q];
    int k = 0;
    for (int t = 1; t < ns; ++t)
      if (load[t] < load[k]) k = t;
    load[k] += work[i];
    cudaStream_t s = pool->s[k];
    const int b = resolve_panel(n[i], panel_b[i], variant);
    const Layout L = make_layout(m[i], n[i], b, variant);
    Work w = bind((char*)workspace + slice * k, L);
    w.status = status + i;
    if (Q[i] != A[i] && cudaMemcpy2DAsync(Q[i], sizeof(double) * lda[i], A[i], sizeof(double) * lda[i],
                                          sizeof(double) * m[i], n[i], cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      rc = CQR_ERR_CUDA;
    else if (cudaMemsetAsync(R[i], 0, sizeof(double) * n[i] * n[i], s) != cudaSuccess)
      rc = CQR_ERR_CUDA;
    else if (factor_run(m[i], n[i], b, Q[i], lda[i], R[i], n[i], variant, w, s) != cudaSuccess)
      rc = CQR_ERR_CUDA;
  }
  // join: the caller's stream waits for every pool stream (also after an error)
  for (int k = 0; k < ns; ++k) {
    if (cudaEventRecord(pool->done[k], pool->s[k]) != cudaSuccess || cudaStreamWaitEvent(st, pool->done[k], 0) != cudaSuccess)
      rc = CQR_ERR_CUDA;
  }
  delete[] order;
  delete[] work;
  return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free factorisation.  Some callers cannot allocate device memory
// at the point where they factor: code running under a fixed memory budget
// planned once at start-up, code called back from inside another
// framework's allocator or memory pool, or code with a rule that nothing
// allocates after initialisation.  For them the scratch that cqr_factor()
// takes as a caller-supplied workspace lives in this file-scope device array
// instead.  Every GPU that loads the library holds it until the process
// exits; under the runtime's lazy module loading it is created on a device
// by the first call there (the symbol lookup below loads the module).
namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[CQR_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};  // device address of g_noalloc_scratch, per device

// First call on a device: look up the array's device address with that
// device current (in host code the array's name is not a device address).
void* noalloc_scratch() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return nullptr;
    g_noalloc_addr[dev] = p;
  }
  return g_noalloc_addr[dev];
}

}  // namespace

int cqr_factor_noalloc(int64_t m, int64_t n, double* A, int64_t lda, int panel_b, double* Q, int64_t ldq, double* R,
                       int64_t ldr, int variant, int* status, cqr_stream_t stream) {
  if (m < 1 || m < n) return -1;
  if (n < 1) return -2;
  if (!A) return -3;
  if (lda < m) return -4;
  if (variant < 0 || variant > 3) return -10;
  if ((variant == CQR_CQR2 || variant == CQR_SCQR3) && n > CQR_MAX_PANEL) return -2;  // one panel, b = n
  const int b = resolve_panel(n, panel_b, variant);
  if (panel_b < 0 || b < 1 || b > CQR_MAX_PANEL || n % b) return -5;
  if (!Q) return -6;
  if (ldq < m || (Q == A && ldq != lda)) return -7;
  if (Q != A && overlaps(A, lda, m, n, Q, ldq)) return -6;
  if (!R) return -8;
  if (ldr < n) return -9;
  const Layout L = make_layout(m, n, b, variant);
  if (L.total > (size_t)CQR_NOALLOC_SCRATCH_BYTES) return CQR_ERR_NOALLOC_TOO_LARGE;
  void* scratch = noalloc_scratch();
  if (!scratch) return CQR_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const Work w = bind(scratch, L);
  cudaGetLastError();
  // The array keeps the previous call's contents: the status word must start at 0.
  if (cudaMemsetAsync(w.status, 0, sizeof(int), st) != cudaSuccess) return CQR_ERR_CUDA;
  if (Q != A && cudaMemcpy2DAsync(Q, sizeof(double) * ldq, A, sizeof(double) * lda, sizeof(double) * m, n,
                                  cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return CQR_ERR_CUDA;
  if (cudaMemset2DAsync(R, sizeof(double) * ldr, 0, sizeof(double) * n, n, st) != cudaSuccess) return CQR_ERR_CUDA;
  if (factor_run(m, n, b, Q, ldq, R, ldr, variant, w, st) != cudaSuccess) return CQR_ERR_CUDA;
  if (status && cudaMemcpyAsync(status, w.status, sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return CQR_ERR_CUDA;
  return 0;
}

const char* cqr_status_string(int status) {
  if (status == 0) return "success";
  if (status == CQR_ERR_NOALLOC_TOO_LARGE)
    return "cqr_factor_noalloc: the factorisation needs more scratch than the fixed CQR_NOALLOC_SCRATCH_BYTES array";
  if (status == CQR_ERR_CUDA) return "a CUDA launch or copy failed";
  if (status == CQR_ERR_ALLOC)
    return "workspace = NULL: the allocator registered with cqr_set_allocator returned no 256-byte aligned memory";
  if (status == CQR_STATUS_TIMEOUT) return "a bounded wait inside a kernel expired";
  if (status > 0) return "Cholesky breakdown: the Gram matrix is not numerically positive definite (status = column + 1)";
  return "invalid argument (status = -(argument position))";
}

double cqr_probe_fp64_peak(int iters) {
  double g = 0.0;
  return probe_fp64(0, iters > 0 ? iters : 20000, &g, nullptr, nullptr) == 0 ? g : -1.0;
}

int cqr_probe_fp64(int kind, int iters, double* gflops, double* flop_per_clk_sm, double* sm_mhz) {
  if (kind < 0 || kind > 2) return -1;
  if (iters < 1) return -2;
  const int rc = probe_fp64(kind, iters, gflops, flop_per_clk_sm, sm_mhz);
  return rc == 0 ? 0 : (rc == -1 ? -2 : CQR_ERR_CUDA);
}

}  // extern "C"
