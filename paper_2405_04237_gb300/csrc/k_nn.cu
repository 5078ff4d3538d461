// C = beta*C + alpha*A*B: the Gram-Schmidt update A_{j:k} -= Q_{j-1} Y
// (Alg. 6 step 7, Alg. 9 step 4), the re-orthogonalisation update
// P -= Q_{1:j-1} Z (Alg. 9 step 7), the blocked part of wide triangular
// solves, the adjoint's Q copyltu(M) product, and the small triangular
// products R = R2 R1 (Alg. 3 step 3, Alg. 7 step 3), R_jj = S2 S1 and
// R_{1:j-1,j} += Z S1 of Alg. 9.
//
// Each block computes a TM x TN output tile (TM * TN = 4096, 256 threads,
// one 4 x 4 register micro-tile per thread); K is staged through shared
// memory in chunks.  With beta = 1 the accumulator starts from C and every
// term is one fused multiply-add (negated operand when alpha = -1), so the
// update issues exactly one FP64 instruction per multiply-add.  Threads
// whose four columns all lie beyond N skip the arithmetic (warp-uniform when
// N is a multiple of 8), so narrow outputs do not pay for padding.
#include "cqr_common.cuh"

namespace cqr {

namespace {

constexpr int kNnThreads = 256;

struct NnArgs {
  const double* A;
  i64 lda;
  const double* B;
  i64 ldb;
  double* C;
  i64 ldc;
  i64 M;
  int N, K;
  int beta, a_upper, b_upper, transb;
  int tiles_n;
  const int* status;
};

template <int TM, int TN>
struct NnShape {
  static constexpr int NTM = TM / 4;
  static constexpr int KC = TM >= 256 ? 8 : 16;
  static constexpr int SA = TM + 2, SB = TN + 2;
  static_assert(TM % 4 == 0 && TN % 4 == 0, "4 x 4 micro-tiles");
  static_assert(NTM * (TN / 4) == kNnThreads, "one micro-tile per thread covers the TM x TN tile");
  static_assert(KC * (SA + SB) * (int)sizeof(double) <= 48 * 1024, "static shared memory limit");
};

template <int TM, int TN, bool NEG>
__global__ void __launch_bounds__(kNnThreads) nn_kernel(NnArgs a) {
  using Sh = NnShape<TM, TN>;
  __shared__ __align__(16) double As[Sh::KC * Sh::SA];
  __shared__ __align__(16) double Bs[Sh::KC * Sh::SB];
  if (a.status && *a.status) return;
  const i64 bid = blockIdx.x;
  const int tn_i = (int)(bid % a.tiles_n);
  const i64 m0 = (bid / a.tiles_n) * TM;
  const int n0 = tn_i * TN;
  const int t = threadIdx.x;
  const int mi = t % Sh::NTM, nj = t / Sh::NTM;
  const bool cols_live = n0 + 4 * nj < a.N;
  const bool rows_live = m0 + 4 * mi < a.M;
  const bool live = cols_live && rows_live;

  int klo = 0, khi = a.K;
  if (a.a_upper) klo = (int)(m0 < (i64)a.K ? m0 : (i64)a.K);
  if (a.b_upper) khi = min(a.K, n0 + TN);

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double v = 0.0;
      if (a.beta) {
        const i64 r = m0 + 4 * mi + i;
        const int c = n0 + 4 * nj + j;
        if (r < a.M && c < a.N) v = a.C[r + (i64)c * a.ldc];
      }
      acc[i][j] = v;
    }

  for (int k0 = klo; k0 < khi; k0 += Sh::KC) {
    for (int e = t; e < Sh::KC * TM; e += kNnThreads) {
      const int mm = e % TM, kk = e / TM;
      const i64 r = m0 + mm;
      const int k = k0 + kk;
      double v = 0.0;
      if (r < a.M && k < khi) v = a.A[r + (i64)k * a.lda];
      As[kk * Sh::SA + mm] = v;
    }
    if (a.transb) {
      for (int e = t; e < Sh::KC * TN; e += kNnThreads) {
        const int nn = e % TN, kk = e / TN;
        const int c = n0 + nn, k = k0 + kk;
        double v = 0.0;
        if (c < a.N && k < khi) v = a.B[c + (i64)k * a.ldb];
        Bs[kk * Sh::SB + nn] = v;
      }
    } else {
      for (int e = t; e < Sh::KC * TN; e += kNnThreads) {
        const int kk = e % Sh::KC, nn = e / Sh::KC;
        const int c = n0 + nn, k = k0 + kk;
        double v = 0.0;
        if (c < a.N && k < khi) v = a.B[k + (i64)c * a.ldb];
        Bs[kk * Sh::SB + nn] = v;
      }
    }
    __syncthreads();
    if (live) {
#pragma unroll 4
      for (int kk = 0; kk < Sh::KC; ++kk) {
        const double2 a01 = *reinterpret_cast<const double2*>(&As[kk * Sh::SA + 4 * mi]);
        const double2 a23 = *reinterpret_cast<const double2*>(&As[kk * Sh::SA + 4 * mi + 2]);
        const double2 b01 = *reinterpret_cast<const double2*>(&Bs[kk * Sh::SB + 4 * nj]);
        const double2 b23 = *reinterpret_cast<const double2*>(&Bs[kk * Sh::SB + 4 * nj + 2]);
        const double av[4] = {a01.x, a01.y, a23.x, a23.y};
        const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = NEG ? fma(-av[i], bv[j], acc[i][j]) : fma(av[i], bv[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const i64 r = m0 + 4 * mi + i;
      const int c = n0 + 4 * nj + j;
      if (r < a.M && c < a.N) a.C[r + (i64)c * a.ldc] = acc[i][j];
    }
}

template <int TM, int TN>
void launch_nn(const NnArgs& a, bool neg, i64 blocks, cudaStream_t st) {
  if (neg)
    nn_kernel<TM, TN, true><<<(unsigned)blocks, kNnThreads, 0, st>>>(a);
  else
    nn_kernel<TM, TN, false><<<(unsigned)blocks, kNnThreads, 0, st>>>(a);
}

}  // namespace

cudaError_t nn_product(i64 M, int N, int K, const double* A, i64 lda, const double* B, i64 ldb, double* C,
                       i64 ldc, double alpha, int beta, int a_upper, int b_upper, const int* status,
                       cudaStream_t st) {
  return nn_product_t(M, N, K, A, lda, B, ldb, 0, C, ldc, alpha, beta, a_upper, b_upper, status, st);
}

cudaError_t nn_product_t(i64 M, int N, int K, const double* A, i64 lda, const double* B, i64 ldb, int transb,
                         double* C, i64 ldc, double alpha, int beta, int a_upper, int b_upper, const int* status,
                         cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  NnArgs a;
  a.A = A;
  a.lda = lda;
  a.B = B;
  a.ldb = ldb;
  a.C = C;
  a.ldc = ldc;
  a.M = M;
  a.N = N;
  a.K = K;
  a.beta = beta;
  a.a_upper = a_upper;
  a.b_upper = b_upper;
  a.transb = transb;
  a.status = status;
  const bool neg = alpha < 0.0;
  int TN = N <= 8 ? 8 : N <= 16 ? 16 : N <= 32 ? 32 : 64;
  int TM = 4096 / TN;
  a.tiles_n = (N + TN - 1) / TN;
  const i64 blocks = ((M + TM - 1) / TM) * a.tiles_n;
  prof_begin(kUpdate, st);
  switch (TN) {
    case 8: launch_nn<512, 8>(a, neg, blocks, st); break;
    case 16: launch_nn<256, 16>(a, neg, blocks, st); break;
    case 32: launch_nn<128, 32>(a, neg, blocks, st); break;
    default: launch_nn<64, 64>(a, neg, blocks, st); break;
  }
  prof_end(kUpdate, 2.0 * (double)M * N * K, st);
  return cudaGetLastError();
}

}  // namespace cqr
