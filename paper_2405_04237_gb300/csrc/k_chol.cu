// One-block Cholesky factorisation W = U^T U of a b x b Gram matrix
// (Alg. 1 step 2; Alg. 2 step 5), right-looking:
//   for j = 0..b-1:  d = W_jj;  breakdown unless d > 0 and finite;
//                    U_jj = sqrt(d);  U_jc = W_jc / U_jj  (c > j);
//                    W_ac -= U_ja U_jc  (j < a <= c).
// Each W_jc receives its updates in ascending j, i.e. the same order as the
// row-by-row definition U_jc = (W_jc - sum_{i<j} U_ij U_ic) / U_jj.
// sqrt and the division are CUDA's correctly rounded double operations.
//
// The b x b problem is a serial island between two streaming passes over
// the m rows; it costs b^3/6 FMAs on one SM (about 90 us for b = 128), a
// few percent of a panel step at the sizes this library targets.  For
// b <= 128 W lives in shared memory (row-major upper triangle); wider
// panels work in place on W in global memory (L2-resident), column-major,
// with the pivot row copied to shared memory each step.
//
// A breakdown (the Gram matrix is not numerically positive definite,
// Sec. 3) sets the status word to col0 + j + 1 with an atomic
// compare-and-swap, so the first breakdown of a factorisation is kept; the
// unfinished rows of U and their reciprocals become NaN.  Nothing traps.
#include "cqr_common.cuh"

namespace cqr {

namespace {

constexpr int kCholThreads = 512;

template <bool SMEM>
__global__ void __launch_bounds__(kCholThreads) chol_kernel(int b, double* W, i64 ldw, double* U, i64 ldu,
                                                            double* rinv, int col0, int* status, int shift, i64 m,
                                                            int* skip, int* reject) {
  extern __shared__ __align__(16) double sm[];
  if (status && *status) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarp = kCholThreads / 32;
  double* urow = sm;            // [b]  pivot row of U
  double* rv = sm + b;          // [b]  reciprocals
  double* Ws = sm + 2 * b;      // [b*b] row-major (SMEM only)
  __shared__ int broken;
  __shared__ int far_from_identity;
  // element (a, c), a <= c
  auto at = [&](int a, int c) -> double& { return SMEM ? Ws[a * b + c] : W[a + (i64)c * ldw]; };
  if (t == 0) {
    broken = -1;
    far_from_identity = 0;
  }
  if (SMEM) {
    for (int e = t; e < b * b; e += kCholThreads) {
      const int a = e % b, c = e / b;
      if (a <= c) Ws[a * b + c] = W[a + (i64)c * ldw];
    }
  }
  __syncthreads();
  if (shift && t == 0) {
    // Alg. 4 steps 2-3: s = sqrt(m) u ||A||_F^2 with ||A||_F^2 = trace(W)
    double fro2 = 0.0;
    for (int j = 0; j < b; ++j) fro2 += at(j, j);
    const double s = sqrt((double)m) * 0x1p-53 * fro2;
    for (int j = 0; j < b; ++j) at(j, j) += s;
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (warp == 0) {
      const double d = at(j, j);
      const bool ok = (d > 0.0) && isfinite(d);
      if (ok) {
        const double u = sqrt(d);
        for (int c = j + 1 + lane; c < b; c += 32) {
          const double v = at(j, c) / u;
          at(j, c) = v;
          urow[c] = v;
        }
        if (lane == 0) {
          at(j, j) = u;
          urow[j] = u;
          rv[j] = 1.0 / u;
        }
      } else if (lane == 0) {
        broken = j;
        // with the panel test of the adaptive width, a breakdown of a panel wider
        // than one column is a rejection, not a failure of the factorisation
        if (status && !(reject && b > 1)) atomicCAS(status, 0, col0 + j + 1);
      }
    }
    __syncthreads();
    if (broken >= 0) break;
    if (SMEM) {
      for (int a = j + 1 + warp; a < b; a += nwarp) {
        const double ua = urow[a];
        for (int c = a + lane; c < b; c += 32) Ws[a * b + c] = fma(-ua, urow[c], Ws[a * b + c]);
      }
    } else {
      for (int c = j + 1 + warp; c < b; c += nwarp) {
        const double uc = urow[c];
        double* col = W + (i64)c * ldw;
        for (int a = j + 1 + lane; a <= c; a += 32) col[a] = fma(-urow[a], uc, col[a]);
      }
    }
    __syncthreads();
  }
  const int jb = broken;
  // Panel test of the adaptive panel width: rejected when the factorisation
  // broke down or (max U_jj / min U_jj)^2 > 1/(64 u); one column never is.
  if (reject && t == 0) {
    int rej = 0;
    if (b > 1) {
      if (jb >= 0) {
        rej = 1;
      } else {
        double dmax = at(0, 0), dmin = at(0, 0);
        for (int j = 1; j < b; ++j) {
          const double d = at(j, j);
          if (d > dmax) dmax = d;
          if (d < dmin) dmin = d;
        }
        rej = dmax * dmax * 64.0 * 0x1p-53 > dmin * dmin;
      }
    }
    *reject = rej;
  }
  // Runtime choice of the second CholeskyQR pass (Sec. 7): when every entry
  // of U - I is within 8u the panel is already orthonormal to working
  // precision; U becomes I exactly and the triangular solve is skipped
  // (with U = I it would leave the panel unchanged).
  bool identity = false;
  if (skip) {
    if (jb < 0) {
      const double tau = 8.0 * 0x1p-53;
      for (int e = t; e < b * b; e += kCholThreads) {
        const int a = e % b, c = e / b;
        if (a <= c && !(fabs(at(a, c) - (a == c ? 1.0 : 0.0)) <= tau)) far_from_identity = 1;
      }
    }
    __syncthreads();
    identity = (jb < 0) && !far_from_identity;
    if (t == 0) *skip = identity ? 1 : 0;
  }
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int e = t; e < b * b; e += kCholThreads) {
    const int a = e % b, c = e / b;
    double v = 0.0;
    if (identity)
      v = (a == c) ? 1.0 : 0.0;
    else if (a <= c)
      v = (jb >= 0 && a >= jb) ? nan : at(a, c);
    U[a + (i64)c * ldu] = v;
  }
  for (int e = t; e < b; e += kCholThreads) rinv[e] = identity ? 1.0 : ((jb >= 0 && e >= jb) ? nan : rv[e]);
}

// M := copyltu(T - G): M_ac = T_ac - G_ac for a >= c, mirrored above.
__global__ void backward_middle_kernel(int n, const double* T, const double* G, double* M) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int a = e % n, c = e / n;
  const int lo = a >= c ? a : c, hi = a >= c ? c : a;  // (lo, hi) in the lower triangle
  M[e] = T[lo + (i64)hi * n] - G[lo + (i64)hi * n];
}

__global__ void diag_reciprocal_kernel(int n, const double* R, i64 ldr, double* rinv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) rinv[j] = 1.0 / R[j + (i64)j * ldr];
}

}  // namespace

cudaError_t chol_factor(int b, double* W, i64 ldw, double* U, i64 ldu, double* rinv, int col0, int* status,
                        int shift_fro, i64 m, cudaStream_t st, int* skip, int* reject) {
  if (b <= 0) return cudaSuccess;
  if (b <= 128) {
    const size_t smem = sizeof(double) * ((size_t)2 * b + (size_t)b * b);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(chol_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(double) * (2 * 128 + 128 * 128)));
      attr = true;
    }
    prof_begin(kCholesky, st);
    chol_kernel<true><<<1, kCholThreads, smem, st>>>(b, W, ldw, U, ldu, rinv, col0, status, shift_fro, m, skip,
                                                     reject);
    prof_end(kCholesky, (double)b * b * b / 3.0, st);
  } else {
    const size_t smem = sizeof(double) * (size_t)2 * b;
    prof_begin(kCholesky, st);
    chol_kernel<false><<<1, kCholThreads, smem, st>>>(b, W, ldw, U, ldu, rinv, col0, status, shift_fro, m, skip,
                                                      reject);
    prof_end(kCholesky, (double)b * b * b / 3.0, st);
  }
  return cudaGetLastError();
}

cudaError_t backward_middle(int n, const double* T, const double* G, double* M, cudaStream_t st) {
  const int thr = 256;
  prof_begin(kMisc, st);
  backward_middle_kernel<<<(n * n + thr - 1) / thr, thr, 0, st>>>(n, T, G, M);
  prof_end(kMisc, (double)n * n, st);
  return cudaGetLastError();
}

cudaError_t diag_reciprocal(int n, const double* R, i64 ldr, double* rinv, cudaStream_t st) {
  prof_begin(kMisc, st);
  diag_reciprocal_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, R, ldr, rinv);
  prof_end(kMisc, (double)n, st);
  return cudaGetLastError();
}

}  // namespace cqr
