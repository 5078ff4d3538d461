// Internal declarations shared by the CUDA translation units of the library.
//
// Every kernel here computes in FP64 on the CUDA-core FMA pipe (DFMA).  On
// GB300 that pipe delivers 2 FP64 FMA per clock per SM (about 1.19 TFLOP/s
// over 152 SMs), while `mma.sync ... .f64` measures slower (about 1.04
// TFLOP/s) and would also waste half of every symmetric Gram product, so the
// tensor cores are not used.  At 2 DFMA per clock an SM consumes only
// about 8 bytes of operands per FMA issued, far under its share of HBM
// bandwidth, so every kernel is bound by the FP64 pipe; the designs aim at
// (a) issuing no FP64 instruction that the algorithm does not need, and
// (b) keeping every SM's pipe busy (single-wave balanced grids, enough
// independent FMA chains per warp).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cqr {

typedef int64_t i64;

__host__ __device__ __forceinline__ i64 imin64(i64 a, i64 b) { return a < b ? a : b; }

// Number of thread blocks a split-m reduction grid aims to keep resident:
// the SM count of GB300.  It only sets how many partial sums exist, so it
// is a constant (not a device query) to keep results reproducible.
constexpr int kSMs = 152;

// ---------------------------------------------------------------------------
// Split-m transposed product  C (p x q) = X^T Y  summed over m rows.
// Stage 1: S persistent blocks split the flattened (output tile, row block)
// items into S equal contiguous ranges and write one partial tile per
// (block, tile) segment.  Stage 2 adds each entry's segments in ascending
// row order.  With sym != 0, X == Y and only entries on or above the
// diagonal are formed (syrk); the reduce mirrors them.
struct TnPlan {
  int tp, tq;        // output tile (8..64; sym: padded width)
  int tiles_p, tiles_q;
  int ntiles;
  int S;             // persistent blocks
  int rb;            // rows per row block
};
TnPlan tn_plan(i64 m, int p, int q, int sym);
size_t tn_partial_doubles(i64 m, int p, int q, int sym);  // S * p * q
// C (ldc) := X^T Y.  `part` must hold tn_partial_doubles() doubles.
cudaError_t tn_product(i64 m, int p, int q, const double* X, i64 ldx, const double* Y, i64 ldy, int sym,
                       double* part, double* C, i64 ldc, const int* status, cudaStream_t st);

// FP64-accurate C = X^T Y on the FP8 tensor cores (k_ozaki.cu): the m-row
// sum of the projections with the Ozaki splitting.  `ws` must hold
// ozaki_workspace_bytes(m, p, q) bytes.
size_t ozaki_workspace_bytes(i64 m, int p, int q);
cudaError_t tn_product_emulated(i64 m, int p, int q, const double* X, i64 ldx, const double* Y, i64 ldy,
                                void* ws, double* C, i64 ldc, const int* status, cudaStream_t st);
// FP64-accurate C (M x N, ldc) -= X (M x K) Y (K x N) on the FP8 tensor
// cores: the m-row updates of the emulated variant.  `ws` must hold
// ozaki_nn_workspace_bytes(M, N, K) bytes.
size_t ozaki_nn_workspace_bytes(i64 M, int N, int K);
cudaError_t nn_update_emulated(i64 M, int N, int K, const double* X, i64 ldx, const double* Y, i64 ldy, double* C,
                               i64 ldc, void* ws, const int* status, cudaStream_t st);

// ---------------------------------------------------------------------------
// C (M x N) = beta*C + alpha * A (M x K) * B (K x N), alpha = +-1, beta in
// {0, 1}.  When beta == 1 the sum starts from C and each term is applied
// with one fused multiply-add in ascending k.  a_upper / b_upper restrict k
// to the nonzero range of an upper-triangular operand.
cudaError_t nn_product(i64 M, int N, int K, const double* A, i64 lda, const double* B, i64 ldb, double* C,
                       i64 ldc, double alpha, int beta, int a_upper, int b_upper, const int* status,
                       cudaStream_t st);
// Same with B read transposed when transb != 0 (B^T stored N x K, ldb).
cudaError_t nn_product_t(i64 M, int N, int K, const double* A, i64 lda, const double* B, i64 ldb, int transb,
                         double* C, i64 ldc, double alpha, int beta, int a_upper, int b_upper, const int* status,
                         cudaStream_t st);

// ---------------------------------------------------------------------------
// One-block Cholesky  W = U^T U (b x b, U upper, positive diagonal).
// Writes U (ldu; strict lower triangle zeroed) and rinv[j] = 1 / U_jj.
// On breakdown at local column j, status is set to col0 + j + 1 (first
// breakdown wins) and U_jj onward are NaN.  `shift_fro` != 0 applies the
// shifted-CholeskyQR shift s = sqrt(m) * 2^-53 * trace(W) first (Alg. 4).
// With `skip` non-null the second-pass rule of the runtime repetition
// choice applies: if every entry of U - I is within 8u, U := I exactly and
// *skip = 1 (else 0).  With `reject` non-null the panel test of the adaptive
// panel width applies: *reject = 1 when b > 1 and the factorisation broke
// down (status then left untouched) or (max U_jj / min U_jj)^2 > 1/(64 u),
// else 0.  The kernel returns early, writing nothing, if *status != 0.
cudaError_t chol_factor(int b, double* W, i64 ldw, double* U, i64 ldu, double* rinv, int col0, int* status,
                        int shift_fro, i64 m, cudaStream_t st, int* skip = nullptr, int* reject = nullptr);

// ---------------------------------------------------------------------------
// Row-wise forward substitution  X := X U^{-1}  (X m x b, b <= kTrsmMaxB),
// using the reciprocals rinv of U's diagonal.  Wider panels are solved in
// blocks of kTrsmMaxB columns with the coupling applied by the GEMM kernel:
// 64 keeps two blocks (eight warps) per SM where a 128-wide tile of rows
// and U would fill the shared memory with one block of four warps
// (b = 128: 0.78 -> 1.13 TFLOP/s on GB300).
constexpr int kTrsmMaxB = 64;
// With `skip` non-null and *skip set on the device, the launch does nothing.
cudaError_t trsm_rows(i64 m, int b, double* X, i64 ldx, const double* U, i64 ldu, const double* rinv,
                      const int* status, cudaStream_t st, const int* skip = nullptr);

// Row-wise back substitution  X := X U^{-T}  (X m x b, b <= kTrsmMaxB): solves
// Abar U^T = B for the adjoint.  rinv as above.
cudaError_t trsm_rows_transposed(i64 m, int b, double* X, i64 ldx, const double* U, i64 ldu,
                                 const double* rinv, cudaStream_t st);

// Adjoint helper: M := copyltu(T - G) for n x n T = R Rbar^T, G = Qbar^T Q
// (all leading dimension n): M_ac = T_ac - G_ac for a >= c, mirrored.
cudaError_t backward_middle(int n, const double* T, const double* G, double* M, cudaStream_t st);
// Reciprocals of the diagonal of R.
cudaError_t diag_reciprocal(int n, const double* R, i64 ldr, double* rinv, cudaStream_t st);

// FP64 throughput probes (k_probe.cu): kind 0 DFMA, 1 mma.sync m8n8k4 .f64,
// 2 mma.sync m16n8k16 .f64.  Synchronous; returns 0 and GFLOP/s, flop per
// clock per SM (from the SM cycle counters) and the effective SM clock.
int probe_fp64(int kind, int iters, double* gflops, double* flop_per_clk_sm, double* sm_mhz);

// ---------------------------------------------------------------------------
// Persistent batched mCQR2GS (k_batched.cu): one cooperative launch over all
// SMs, groups of G CTAs factoring whole matrices (n <= 128, n and b
// multiples of 4).  `halve` applies the adaptive panel width on the device.
bool batched_persistent_eligible(int batch, const int64_t* m, const int64_t* n, const int* b);
size_t batched_persistent_workspace(int batch);
int batched_persistent_grid();  // CTAs of the launch: one per SM
cudaError_t batched_persistent_run(int batch, const int64_t* m, const int64_t* n, const int64_t* lda,
                                   const int* b, double* const* A, double* const* Q, double* const* R,
                                   int* status, void* workspace, int G, bool halve, cudaStream_t st);
cudaError_t batched_persistent_panels(int batch, const void* workspace, int* host_b, cudaStream_t st);

// ---------------------------------------------------------------------------
// Launch accounting (prof.cu).  Every launch is wrapped in prof_begin /
// prof_end with its kernel class and algorithmic FLOP count.
enum KernelClass {
  kGram = 0,       // syrk partials of W = X^T X
  kProjection = 1, // split-m partials of Y = X^T Z
  kReduce = 2,     // fixed-order sums of split-m partials
  kCholesky = 3,
  kTrsm = 4,
  kUpdate = 5,     // C = beta C + alpha A B (GS / re-orthogonalisation updates, R products)
  kMisc = 6,       // adjoint helpers, probes, digit splitting of the emulated products
  kBatched = 7,
  kNumClasses = 8
};
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, double flops, cudaStream_t st);

// Phase ranges of the host-side enqueue (prof.cu): an NVTX range in the
// domain "cqr" and, when registered, the cqr_set_trace callback, for the
// lifetime of the object.  `name` must be a string literal.
struct TracePhase {
  TracePhase(const char* name, int panel);
  ~TracePhase();
  TracePhase(const TracePhase&) = delete;
  TracePhase& operator=(const TracePhase&) = delete;
  const char* name;
  int panel;
};

}  // namespace cqr
