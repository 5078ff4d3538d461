// Split-m transposed products: the Gram matrix W = X^T X (Alg. 1 step 1,
// syrk semantics as in the caption of Table 1) and the projections
// Y = Q^T A (Alg. 6 step 6, Alg. 9 steps 3 and 7).
//
// The m-row sum is the "Gram reduce" of Alg. 2 step 4 / Alg. 8 steps 3 and 8,
// done inside one GPU: persistent thread blocks each own a contiguous range
// of (output tile, row block) work items, write one partial tile per
// (block, tile) segment, and a second kernel adds the partials in ascending
// row order.  The item ranges are static, so the summation order -- and the
// result -- is the same on every run.
//
// Each thread owns a 4 x 4 micro-tile of the output and, per row, issues 16
// FP64 FMAs on operands staged in shared memory (row-major, padded).  For
// small outputs several thread groups split the rows of a block and are
// summed in group order at the end.
#include "cqr_common.cuh"

namespace cqr {

namespace {

constexpr int kTnThreads = 256;
constexpr int kSyrkThreads = 512;  // 16 warps
// Persistent blocks per SM for the split-m grids (at most what the
// registers allow).  Each block stalls in the load burst at the start of a
// row block; with three resident blocks the others keep the FP64 pipe busy
// meanwhile (projection: 1.195 -> 1.213 TFLOP/s on GB300 against two).
constexpr int kMaxResident = 3;

// Upper-triangle enumeration, column by column: u -> (i, j), 0 <= i <= j.
__host__ __device__ inline void decode_upper(int u, int& i, int& j) {
  int jj = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
  while ((jj + 1) * (jj + 2) / 2 <= u) ++jj;
  while (jj * (jj + 1) / 2 > u) --jj;
  j = jj;
  i = u - jj * (jj + 1) / 2;
}

// [begin, end) of the items of persistent block c when T items are split
// over P blocks.
__host__ __device__ inline void item_range(i64 c, i64 T, i64 P, i64& begin, i64& end) {
  begin = (c * T) / P;
  end = ((c + 1) * T) / P;
}
// The persistent block whose range contains item i.
__host__ __device__ inline i64 owner_of(i64 i, i64 T, i64 P) { return ((i + 1) * P - 1) / T; }

__device__ inline double2 lds2(const double* p) { return *reinterpret_cast<const double2*>(p); }

// ---------------------------------------------------------------------------
// Gram (syrk) kernel for b <= 128, 512 threads (16 warps: four per warp
// scheduler, so every scheduler's share of the FP64 pipe gets the same
// work).  The upper triangle is cut into cnt = T(T+1)/2 tiles of 4 x 4
// (T = ceil(b/4)).  The largest power of two M <= cnt of them are "main"
// tiles: thread t owns main tile t % M on the rows r = t / M (mod 512 / M)
// of each staged row block.  The E = cnt - M other tiles are "extra": each
// is owned by 512 / E threads (whole warps when E <= 16) that split the
// rows round-robin.  Every thread thus carries one main and at most one
// extra accumulator and runs the same instruction stream as its warp.
struct SyrkArgs {
  const double* X;
  i64 ldx, m;
  int b, bp;       // width, padded width (multiple of 4)
  int M, RG;       // main tiles, row groups
  int E, tpt;      // extra tiles, threads per extra tile
  int rb;          // rows per block
  i64 nb, P;       // row blocks, persistent blocks
  double* part;    // [P][b*b]
  const int* status;
};

__device__ __forceinline__ void syrk_tile_row(const double* row, int i, int j, double (&acc)[4][4]) {
  const double2 p0 = lds2(row + 4 * i), p1 = lds2(row + 4 * i + 2);
  const double2 q0 = lds2(row + 4 * j), q1 = lds2(row + 4 * j + 2);
  const double xv[4] = {p0.x, p0.y, p1.x, p1.y};
  const double yv[4] = {q0.x, q0.y, q1.x, q1.y};
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = fma(xv[u], yv[v], acc[u][v]);
}

__device__ __forceinline__ void syrk_store_tile(double* P, int b, int i, int j, const double (&v)[4][4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int r = 4 * i + u, c = 4 * j + w;
      if (r <= c && c < b) P[r + c * b] = v[u][w];
    }
}

__global__ void __launch_bounds__(kSyrkThreads) syrk_partial_kernel(SyrkArgs a) {
  extern __shared__ __align__(16) double sm[];
  if (a.status && *a.status) return;
  const int t = threadIdx.x;
  const int sp = a.bp + 2;  // padded row stride (even: keeps 16-byte alignment)
  int mi, mj;
  decode_upper(t % a.M, mi, mj);
  const int g = t / a.M;
  const bool extra = a.E > 0 && t < a.E * a.tpt;
  int ei = 0, ej = 0;
  const int ek = extra ? t % a.tpt : 0;
  if (extra) decode_upper(a.M + t / a.tpt, ei, ej);
  double am[4][4], ae[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) am[u][v] = ae[u][v] = 0.0;

  i64 ib, ie;
  item_range(blockIdx.x, a.nb, a.P, ib, ie);
  const int rb = a.rb;
  for (i64 blk = ib; blk < ie; ++blk) {
    const i64 r0 = blk * rb;
    const int nrow = (int)imin64(rb, a.m - r0);
    // stage X[r0:r0+rb, 0:bp] row-major; zero beyond m and beyond b.
    // Asynchronous copies: every load of the block is in flight before the
    // one wait, instead of one memory latency per loop iteration.
    for (int e = t; e < rb * a.bp; e += kSyrkThreads) {
      const int r = e % rb, c = e / rb;
      const bool ok = r < nrow && c < a.b;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(sm + r * sp + c);
      const double* src = ok ? a.X + (r0 + r) + (i64)c * a.ldx : a.X;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(ok ? 8 : 0) : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
#pragma unroll 2
    for (int r = g; r < nrow; r += a.RG) syrk_tile_row(sm + r * sp, mi, mj, am);
    if (extra)
      for (int r = ek; r < nrow; r += a.tpt) syrk_tile_row(sm + r * sp, ei, ej, ae);
    __syncthreads();
  }
  // fixed-order sums: main tiles over the row groups, extra tiles over their threads
  double* P = a.part + (i64)blockIdx.x * a.b * a.b;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) sm[(u * 4 + v) * kSyrkThreads + t] = am[u][v];
  __syncthreads();
  if (t < a.M) {
    double sum[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double x = 0.0;
        for (int gg = 0; gg < a.RG; ++gg) x += sm[(u * 4 + v) * kSyrkThreads + gg * a.M + t];
        sum[u][v] = x;
      }
    syrk_store_tile(P, a.b, mi, mj, sum);
  }
  if (a.E > 0) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) sm[(u * 4 + v) * kSyrkThreads + t] = ae[u][v];
    __syncthreads();
    if (extra && ek == 0) {
      double sum[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          double x = 0.0;
          for (int k = 0; k < a.tpt; ++k) x += sm[(u * 4 + v) * kSyrkThreads + t + k];
          sum[u][v] = x;
        }
      syrk_store_tile(P, a.b, ei, ej, sum);
    }
  }
}

// W[r + c*ldw] = sum_{s<P} part[s][r + c*b] for r <= c, mirrored.
__global__ void syrk_reduce_kernel(const double* part, int b, i64 P, double* W, i64 ldw, const int* status) {
  if (status && *status) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= b * b) return;
  const int r = e % b, c = e / b;
  if (r > c) return;
  double s = 0.0;
  for (i64 k = 0; k < P; ++k) s += part[k * b * b + e];
  W[r + (i64)c * ldw] = s;
  if (r != c) W[c + (i64)r * ldw] = s;
}

// ---------------------------------------------------------------------------
// General C = X^T Y (no symmetry).  Tile TP x TQ, 256 threads.
struct TnArgs {
  const double* X;
  i64 ldx;
  const double* Y;
  i64 ldy;
  i64 m;
  int p, q;
  int tiles_p;
  i64 nb, T, P;  // row blocks per tile, total items, persistent blocks
  double* part;  // [P + ntiles][TP*TQ]
  const int* status;
};

template <int TP, int TQ>
struct TnShape {
  static constexpr int NP = TP / 4, NQ = TQ / 4;
  static constexpr int NTG = NP * NQ;
  static constexpr int G = kTnThreads / NTG;
  static constexpr int RB0 = 4096 / (TP + TQ);
  static constexpr int UNIT = G > 8 ? G : 8;
  static constexpr int RB = (RB0 / UNIT) * UNIT;
  static constexpr int SP = TP + 2, SQ = TQ + 2;
  static constexpr int TILE_D = RB * (SP + SQ);
  static constexpr int RED_D = 16 * kTnThreads;
  static constexpr int SMEM_D = TILE_D > RED_D ? TILE_D : RED_D;
  static_assert(TP % 4 == 0 && TQ % 4 == 0, "4 x 4 micro-tiles");
  static_assert(NTG * G == kTnThreads, "every thread owns one micro-tile of one row group");
  static_assert(RB >= G, "every row group gets rows");
  static_assert(SMEM_D * (int)sizeof(double) <= 48 * 1024, "static shared memory limit");
};

template <int TP, int TQ>
__global__ void __launch_bounds__(kTnThreads) tn_partial_kernel(TnArgs a) {
  using Sh = TnShape<TP, TQ>;
  __shared__ __align__(16) double sm[Sh::SMEM_D];
  if (a.status && *a.status) return;
  const int t = threadIdx.x;
  const int g = t / Sh::NTG, u = t - g * Sh::NTG;
  const int mi = u % Sh::NP, mj = u / Sh::NP;
  double* Xs = sm;
  double* Ys = sm + Sh::RB * Sh::SP;

  i64 ib, ie;
  item_range(blockIdx.x, a.T, a.P, ib, ie);
  i64 item = ib;
  while (item < ie) {
    const i64 tile = item / a.nb;
    const i64 tile_end = imin64(ie, (tile + 1) * a.nb);
    const int p0 = (int)(tile % a.tiles_p) * TP, q0 = (int)(tile / a.tiles_p) * TQ;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (; item < tile_end; ++item) {
      const i64 r0 = (item - tile * a.nb) * Sh::RB;
      const int nrow = (int)imin64(Sh::RB, a.m - r0);
      // asynchronous staging (zero-filled beyond m, p, q): all loads in flight before one wait
      for (int e = t; e < Sh::RB * TP; e += kTnThreads) {
        const int r = e % Sh::RB, c = e / Sh::RB;
        const bool ok = r < nrow && p0 + c < a.p;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(Xs + r * Sh::SP + c);
        const double* src = ok ? a.X + (r0 + r) + (i64)(p0 + c) * a.ldx : a.X;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(ok ? 8 : 0) : "memory");
      }
      for (int e = t; e < Sh::RB * TQ; e += kTnThreads) {
        const int r = e % Sh::RB, c = e / Sh::RB;
        const bool ok = r < nrow && q0 + c < a.q;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(Ys + r * Sh::SQ + c);
        const double* src = ok ? a.Y + (r0 + r) + (i64)(q0 + c) * a.ldy : a.Y;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(ok ? 8 : 0) : "memory");
      }
      asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
      __syncthreads();
      const double* xi = Xs + 4 * mi;
      const double* yj = Ys + 4 * mj;
#pragma unroll 2
      for (int r = g; r < nrow; r += Sh::G) {
        const double2 p0v = lds2(xi + r * Sh::SP), p1v = lds2(xi + r * Sh::SP + 2);
        const double2 q0v = lds2(yj + r * Sh::SQ), q1v = lds2(yj + r * Sh::SQ + 2);
        const double xv[4] = {p0v.x, p0v.y, p1v.x, p1v.y};
        const double yv[4] = {q0v.x, q0v.y, q1v.x, q1v.y};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(xv[i], yv[j], acc[i][j]);
      }
      __syncthreads();
    }
    if (Sh::G > 1) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sm[(i * 4 + j) * kTnThreads + t] = acc[i][j];
      __syncthreads();
      if (g == 0) {
        for (int gg = 1; gg < Sh::G; ++gg) {
          const int tt = gg * Sh::NTG + u;
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += sm[(i * 4 + j) * kTnThreads + tt];
        }
      }
      __syncthreads();
    }
    if (g == 0) {
      // segment id = persistent block + tile (unique, increasing in rows)
      double* Pp = a.part + ((i64)blockIdx.x + tile) * (TP * TQ);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Pp[(4 * mi + i) + (4 * mj + j) * TP] = acc[i][j];
    }
  }
}

// C[r + c*ldc] = sum over the segments of tile(r, c), ascending rows.
__global__ void tn_reduce_kernel(const double* part, int p, int q, int TP, int TQ, int tiles_p, i64 nb, i64 T,
                                 i64 P, double* C, i64 ldc, const int* status) {
  if (status && *status) return;
  const i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (i64)p * q) return;
  const int r = (int)(e % p), c = (int)(e / p);
  if (T == 0) {  // no rows: the empty sum
    C[r + (i64)c * ldc] = 0.0;
    return;
  }
  const i64 tile = (i64)(r / TP) + (i64)(c / TQ) * tiles_p;
  const int loc = (r % TP) + (c % TQ) * TP;
  const i64 c_lo = owner_of(tile * nb, T, P);
  const i64 c_hi = owner_of((tile + 1) * nb - 1, T, P);
  double s = 0.0;
  for (i64 blk = c_lo; blk <= c_hi; ++blk) s += part[(blk + tile) * (TP * TQ) + loc];
  C[r + (i64)c * ldc] = s;
}

// ---------------------------------------------------------------------------
inline int pick_tile(int d) { return d <= 8 ? 8 : d <= 16 ? 16 : d <= 32 ? 32 : 64; }

struct SyrkPlan {
  int bp, M, RG, E, tpt, rb;
  size_t smem;
};
SyrkPlan syrk_plan(int b) {
  SyrkPlan s;
  const int n4 = (b + 3) / 4;
  s.bp = 4 * n4;
  const int cnt = n4 * (n4 + 1) / 2;
  s.M = 1;
  while (s.M * 2 <= cnt && s.M * 2 <= kSyrkThreads) s.M *= 2;
  s.RG = kSyrkThreads / s.M;
  s.E = cnt - s.M;
  s.tpt = s.E > 0 ? kSyrkThreads / s.E : 0;
  // about 8192 staged doubles (the size of the reduction area) per row
  // block, a multiple of the row groups
  const int per = 8192 / (s.bp + 2);
  s.rb = per >= s.RG ? per / s.RG * s.RG : s.RG;
  const size_t tile = (size_t)s.rb * (s.bp + 2), red = (size_t)16 * kSyrkThreads;
  s.smem = (tile > red ? tile : red) * sizeof(double);
  return s;
}

int g_occ_syrk[129];
int g_occ_tn[4][4];

int syrk_occupancy(int b, const SyrkPlan& s) {
  if (g_occ_syrk[b] == 0) {
    cudaFuncSetAttribute(syrk_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, syrk_partial_kernel, kSyrkThreads, s.smem);
    g_occ_syrk[b] = occ > 0 ? occ : 1;
  }
  return g_occ_syrk[b];
}

template <int TP, int TQ>
int tn_occ_impl() {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tn_partial_kernel<TP, TQ>, kTnThreads, 0);
  return occ > 0 ? occ : 1;
}
inline int tidx(int t) { return t == 8 ? 0 : t == 16 ? 1 : t == 32 ? 2 : 3; }

template <int TP>
int tn_occ_q(int tq) {
  switch (tq) {
    case 8: return tn_occ_impl<TP, 8>();
    case 16: return tn_occ_impl<TP, 16>();
    case 32: return tn_occ_impl<TP, 32>();
    default: return tn_occ_impl<TP, 64>();
  }
}
int tn_occupancy(int tp, int tq) {
  int& o = g_occ_tn[tidx(tp)][tidx(tq)];
  if (o == 0) {
    switch (tp) {
      case 8: o = tn_occ_q<8>(tq); break;
      case 16: o = tn_occ_q<16>(tq); break;
      case 32: o = tn_occ_q<32>(tq); break;
      default: o = tn_occ_q<64>(tq); break;
    }
  }
  return o;
}

int tn_rb(int tp, int tq) {
  const int ntg = (tp / 4) * (tq / 4);
  const int G = kTnThreads / ntg;
  const int unit = G > 8 ? G : 8;
  return ((4096 / (tp + tq)) / unit) * unit;
}

template <int TP>
void launch_tn_q(int tq, dim3 grid, cudaStream_t st, const TnArgs& a) {
  switch (tq) {
    case 8: tn_partial_kernel<TP, 8><<<grid, kTnThreads, 0, st>>>(a); break;
    case 16: tn_partial_kernel<TP, 16><<<grid, kTnThreads, 0, st>>>(a); break;
    case 32: tn_partial_kernel<TP, 32><<<grid, kTnThreads, 0, st>>>(a); break;
    default: tn_partial_kernel<TP, 64><<<grid, kTnThreads, 0, st>>>(a); break;
  }
}

}  // namespace

TnPlan tn_plan(i64 m, int p, int q, int sym) {
  TnPlan P{};
  if (sym && p <= 128) {
    SyrkPlan s = syrk_plan(p);
    P.tp = P.tq = s.bp;
    P.tiles_p = P.tiles_q = 1;
    P.ntiles = 1;
    P.rb = s.rb;
    const i64 nb = (m + s.rb - 1) / s.rb;
    i64 slots = (i64)kSMs * min(syrk_occupancy(p, s), kMaxResident);
    P.S = (int)(nb < slots ? (nb > 0 ? nb : 1) : slots);
    return P;
  }
  P.tp = pick_tile(p);
  P.tq = pick_tile(q);
  P.tiles_p = (p + P.tp - 1) / P.tp;
  P.tiles_q = (q + P.tq - 1) / P.tq;
  P.ntiles = P.tiles_p * P.tiles_q;
  P.rb = tn_rb(P.tp, P.tq);
  const i64 nb = (m + P.rb - 1) / P.rb;
  const i64 T = nb * P.ntiles;
  i64 slots = (i64)kSMs * min(tn_occupancy(P.tp, P.tq), kMaxResident);
  P.S = (int)(T < slots ? (T > 0 ? T : 1) : slots);
  return P;
}

size_t tn_partial_doubles(i64 m, int p, int q, int sym) {
  if (p <= 0 || q <= 0) return 0;
  if (sym && p > 128) {
    // blocked into 128-wide pieces: the largest piece dominates
    size_t mx = 0;
    for (int i = 0; i < p; i += 128)
      for (int j = i; j < p; j += 128) {
        int pi = p - i < 128 ? p - i : 128, pj = p - j < 128 ? p - j : 128;
        size_t d = tn_partial_doubles(m, pi, pj, i == j);
        if (d > mx) mx = d;
      }
    return mx;
  }
  TnPlan P = tn_plan(m, p, q, sym);
  if (sym) return (size_t)P.S * p * p;
  return (size_t)(P.S + P.ntiles) * P.tp * P.tq;
}

cudaError_t tn_product(i64 m, int p, int q, const double* X, i64 ldx, const double* Y, i64 ldy, int sym,
                       double* part, double* C, i64 ldc, const int* status, cudaStream_t st) {
  if (p <= 0 || q <= 0) return cudaSuccess;
  if (sym && p > 128) {
    // W = [X1 X2 ...]^T [X1 X2 ...] by 128-wide blocks; upper blocks, mirrored.
    for (int j = 0; j < p; j += 128) {
      for (int i = 0; i <= j; i += 128) {
        const int pi = p - i < 128 ? p - i : 128, pj = p - j < 128 ? p - j : 128;
        cudaError_t e;
        if (i == j) {
          e = tn_product(m, pi, pi, X + (i64)i * ldx, ldx, X + (i64)i * ldx, ldx, 1, part, C + i + (i64)i * ldc,
                         ldc, status, st);
        } else {
          e = tn_product(m, pi, pj, X + (i64)i * ldx, ldx, X + (i64)j * ldx, ldx, 0, part, C + i + (i64)j * ldc,
                         ldc, status, st);
        }
        if (e != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  }
  TnPlan P = tn_plan(m, p, q, sym);
  if (sym) {
    SyrkPlan s = syrk_plan(p);
    SyrkArgs a;
    a.X = X;
    a.ldx = ldx;
    a.m = m;
    a.b = p;
    a.bp = s.bp;
    a.M = s.M;
    a.RG = s.RG;
    a.E = s.E;
    a.tpt = s.tpt;
    a.rb = s.rb;
    a.nb = (m + s.rb - 1) / s.rb;
    a.P = P.S;
    a.part = part;
    a.status = status;
    if (m > 0) {
      prof_begin(kGram, st);
      syrk_partial_kernel<<<P.S, kSyrkThreads, s.smem, st>>>(a);
      prof_end(kGram, (double)m * p * (p + 1), st);
    }
    const int thr = 256;
    const int blocks = (p * p + thr - 1) / thr;
    const i64 nsum = m > 0 ? P.S : 0;  // m == 0: the empty sum, W = 0
    prof_begin(kReduce, st);
    syrk_reduce_kernel<<<blocks, thr, 0, st>>>(part, p, nsum, C, ldc, status);
    prof_end(kReduce, (double)nsum * p * (p + 1) / 2, st);
    return cudaGetLastError();
  }
  TnArgs a;
  a.X = X;
  a.ldx = ldx;
  a.Y = Y;
  a.ldy = ldy;
  a.m = m;
  a.p = p;
  a.q = q;
  a.tiles_p = P.tiles_p;
  a.nb = (m + P.rb - 1) / P.rb;
  a.T = a.nb * P.ntiles;
  a.P = P.S;
  a.part = part;
  a.status = status;
  if (m > 0) {
    dim3 grid((unsigned)P.S);
    prof_begin(kProjection, st);
    switch (P.tp) {
      case 8: launch_tn_q<8>(P.tq, grid, st, a); break;
      case 16: launch_tn_q<16>(P.tq, grid, st, a); break;
      case 32: launch_tn_q<32>(P.tq, grid, st, a); break;
      default: launch_tn_q<64>(P.tq, grid, st, a); break;
    }
    prof_end(kProjection, 2.0 * (double)m * p * q, st);
  }
  const i64 pq = (i64)p * q;
  const int thr = 256;
  const unsigned blocks = (unsigned)((pq + thr - 1) / thr);
  prof_begin(kReduce, st);
  tn_reduce_kernel<<<blocks, thr, 0, st>>>(part, p, q, P.tp, P.tq, P.tiles_p, a.nb, m > 0 ? a.T : 0,
                                           m > 0 ? a.P : 1, C, ldc, status);
  prof_end(kReduce, m > 0 ? (double)(P.S + P.ntiles) / P.ntiles * pq : 0.0, st);
  return cudaGetLastError();
}

}  // namespace cqr
