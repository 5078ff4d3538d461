// Row-wise triangular solves.
//
// trsm_rows: Q = X U^{-1} (Alg. 1 step 3).  Every row x of X is solved by
// forward substitution, q_c = (x_c - sum_{i<c} q_i U_ic) * (1/U_cc), the
// sum taken in ascending i -- the same operation order as the plain
// definition, with the division replaced by a multiplication by the
// reciprocal that the Cholesky kernel computed once (a division costs about
// ten FP64 instructions; the substitution itself costs b(b-1)/2 FMAs per
// row).  No inverse of U is formed: substitution keeps each row backward
// stable, so the residual ||A - Q R|| stays at rounding level even when U
// is ill-conditioned.
//
// trsm_rows_transposed: Abar = B U^{-T} for the adjoint of A = QR, by back
// substitution a_c = (b_c - sum_{i>c} a_i U_ci) * (1/U_cc), descending c.
//
// One thread owns one row; 128 rows per block.  The rows live in shared
// memory, column-major in the row index (conflict-free), and U's upper
// triangle is packed row by row in shared memory (every thread reads the
// same U entry: a broadcast).  Columns are solved in groups of sixteen so
// that each warp keeps sixteen independent FMA chains in flight: with one
// block of four warps per SM (b = 128 needs 194 KB of shared memory) fewer
// chains leave the FP64 pipe waiting on dependent FMAs.
#include "cqr_common.cuh"

namespace cqr {

namespace {

constexpr int kRows = 128;
constexpr int kGrp = 16;

__device__ __forceinline__ int packed_off(int i, int b) { return i * b - (i * (i - 1)) / 2; }

// shared memory: tile [b][kRows], packed U (b(b+1)/2 + kGrp pad), rinv[b]
inline size_t trsm_smem(int b) {
  return sizeof(double) * ((size_t)b * kRows + (size_t)b * (b + 1) / 2 + kGrp + b);
}

// 8-byte asynchronous global -> shared copy (all of a block's staging loads
// in flight before one wait, instead of one memory latency per iteration).
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void load_common(int b, const double* U, i64 ldu, const double* rinv, double* Up,
                                            double* rv) {
  const int t = threadIdx.x;
  for (int e = t; e < b * b; e += kRows) {
    const int i = e % b, c = e / b;
    if (i <= c) Up[packed_off(i, b) + c - i] = U[i + (i64)c * ldu];
  }
  if (t < kGrp) Up[b * (b + 1) / 2 + t] = 0.0;
  for (int e = t; e < b; e += kRows) rv[e] = rinv[e];
}

__global__ void __launch_bounds__(kRows) trsm_rows_kernel(i64 m, int b, double* X, i64 ldx, const double* U, i64 ldu,
                                                          const double* rinv, const int* status, const int* skip) {
  extern __shared__ __align__(16) double sm[];
  if (status && *status) return;
  if (skip && *skip) return;  // U = I: the solve would leave X unchanged
  double* Ts = sm;
  double* Up = sm + (size_t)b * kRows;
  double* rv = Up + b * (b + 1) / 2 + kGrp;
  const int t = threadIdx.x;
  const i64 r0 = (i64)blockIdx.x * kRows;
  const int nrow = (int)imin64(kRows, m - r0);
  if (t < nrow)
    for (int c = 0; c < b; ++c) cp_async8(Ts + c * kRows + t, X + r0 + t + (i64)c * ldx);
  load_common(b, U, ldu, rinv, Up, rv);
  cp_async_wait_all();
  __syncthreads();
  if (t < nrow) {
    for (int g0 = 0; g0 < b; g0 += kGrp) {
      double s[kGrp];
#pragma unroll
      for (int k = 0; k < kGrp; ++k) s[k] = (g0 + k < b) ? Ts[(g0 + k) * kRows + t] : 0.0;
      // contributions of the already solved columns, ascending i
#pragma unroll 2
      for (int i = 0; i < g0; ++i) {
        const double q = Ts[i * kRows + t];
        const double* u = Up + packed_off(i, b) + (g0 - i);
#pragma unroll
        for (int k = 0; k < kGrp; ++k) s[k] = fma(-q, u[k], s[k]);
      }
      // substitution inside the group
#pragma unroll
      for (int k = 0; k < kGrp; ++k) {
        if (g0 + k < b) {
          const double q = s[k] * rv[g0 + k];
          Ts[(g0 + k) * kRows + t] = q;
          const double* u = Up + packed_off(g0 + k, b);
#pragma unroll
          for (int k2 = k + 1; k2 < kGrp; ++k2) s[k2] = fma(-q, u[k2 - k], s[k2]);
        }
      }
    }
    for (int c = 0; c < b; ++c) X[r0 + t + (i64)c * ldx] = Ts[c * kRows + t];
  }
}

__global__ void __launch_bounds__(kRows) trsm_rows_t_kernel(i64 m, int b, double* X, i64 ldx, const double* U, i64 ldu,
                                                            const double* rinv) {
  extern __shared__ __align__(16) double sm[];
  double* Ts = sm;
  double* Up = sm + (size_t)b * kRows;
  double* rv = Up + b * (b + 1) / 2 + kGrp;
  const int t = threadIdx.x;
  const i64 r0 = (i64)blockIdx.x * kRows;
  const int nrow = (int)imin64(kRows, m - r0);
  if (t < nrow)
    for (int c = 0; c < b; ++c) cp_async8(Ts + c * kRows + t, X + r0 + t + (i64)c * ldx);
  load_common(b, U, ldu, rinv, Up, rv);
  cp_async_wait_all();
  __syncthreads();
  if (t < nrow) {
    // groups [g_lo, g_hi) from the right; s[k] holds column g_hi-1-k
    for (int g_hi = b; g_hi > 0; g_hi -= kGrp) {
      double s[kGrp];
#pragma unroll
      for (int k = 0; k < kGrp; ++k) s[k] = (g_hi - 1 - k >= 0) ? Ts[(g_hi - 1 - k) * kRows + t] : 0.0;
      // contributions of the solved columns i >= g_hi, in ascending i
      for (int i = g_hi; i < b; ++i) {
        const double av = Ts[i * kRows + t];
#pragma unroll
        for (int k = 0; k < kGrp; ++k) {
          const int c = g_hi - 1 - k;
          if (c >= 0) s[k] = fma(-av, Up[packed_off(c, b) + (i - c)], s[k]);
        }
      }
      // back substitution inside the group: c = g_hi-1, g_hi-2, ...
#pragma unroll
      for (int k = 0; k < kGrp; ++k) {
        const int c = g_hi - 1 - k;
        if (c >= 0) {
          const double av = s[k] * rv[c];
          Ts[c * kRows + t] = av;
#pragma unroll
          for (int k2 = k + 1; k2 < kGrp; ++k2) {
            const int c2 = g_hi - 1 - k2;
            if (c2 >= 0) s[k2] = fma(-av, Up[packed_off(c2, b) + (c - c2)], s[k2]);
          }
        }
      }
    }
    for (int c = 0; c < b; ++c) X[r0 + t + (i64)c * ldx] = Ts[c * kRows + t];
  }
}

bool g_trsm_attr = false;
void set_trsm_attr() {
  if (!g_trsm_attr) {
    const int mx = (int)trsm_smem(kTrsmMaxB);
    cudaFuncSetAttribute(trsm_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(trsm_rows_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    g_trsm_attr = true;
  }
}

}  // namespace

cudaError_t trsm_rows(i64 m, int b, double* X, i64 ldx, const double* U, i64 ldu, const double* rinv,
                      const int* status, cudaStream_t st, const int* skip) {
  if (m <= 0 || b <= 0) return cudaSuccess;
  if (b > kTrsmMaxB) return cudaErrorInvalidValue;
  set_trsm_attr();
  const i64 blocks = (m + kRows - 1) / kRows;
  prof_begin(kTrsm, st);
  trsm_rows_kernel<<<(unsigned)blocks, kRows, trsm_smem(b), st>>>(m, b, X, ldx, U, ldu, rinv, status, skip);
  prof_end(kTrsm, (double)m * b * b, st);
  return cudaGetLastError();
}

cudaError_t trsm_rows_transposed(i64 m, int b, double* X, i64 ldx, const double* U, i64 ldu,
                                 const double* rinv, cudaStream_t st) {
  if (m <= 0 || b <= 0) return cudaSuccess;
  if (b > kTrsmMaxB) return cudaErrorInvalidValue;
  set_trsm_attr();
  const i64 blocks = (m + kRows - 1) / kRows;
  prof_begin(kTrsm, st);
  trsm_rows_t_kernel<<<(unsigned)blocks, kRows, trsm_smem(b), st>>>(m, b, X, ldx, U, ldu, rinv);
  prof_end(kTrsm, (double)m * b * b, st);
  return cudaGetLastError();
}

}  // namespace cqr
