// FP64-accurate split-m products C = X^T Y on the FP8 tensor cores (the
// Ozaki error-free splitting; Ozaki, Ogita, Oishi, Numer. Algorithms 59
// (2012)), for the emulated variant of the projections of Alg. 9 steps 3
// and 7 (opt-in, CQR_EMULATED).
//
// Splitting.  Rows are cut into sub-chunks of kSub = 4096.  Within a
// sub-chunk every column c of X (and of Y) gets a power-of-two scale 2^e_c
// with |x| < 2^(e_c - 1), and each entry becomes the 56-bit fixed-point
// integer |x| * 2^(56 - e_c) (truncated below 2^-56 of the scale) split into
// 14 unsigned nibbles n_0..n_13 (n_i has weight 16^i); digit i of x is
// sign(x) * n_i, an integer in [-15, 15] that e4m3 represents exactly.
// Digits live in 14 "planes" laid out [sub-chunk][32-row stage][plane]
// [column][32 bytes], so that one stage of a 32-column tile is 14
// contiguous 1 KiB runs per operand.
//
// Products.  x_a y_b = 2^(e_a + e_b - 112) sum_{i,j} d^x_i d^y_j 16^(i+j).
// The 105 plane pairs with i + j >= 13 (the 14 most significant weight
// levels) are multiplied with mma.sync m16n8k32 e4m3 -> f32.  Per level the
// sum over a sub-chunk is at most 14 * 225 * 4096 < 2^24 in magnitude, so
// the FP32 accumulation is exact (an integer).  The dropped levels weigh at
// most about 2^-52 of the column scales' product per row.
//
// Schedule.  A block (7 warps) computes a 32 x 32 tile of C for one
// sub-chunk: warp w owns levels 13 + w and 26 - w (15 plane pairs, equal for
// every warp); the planes of 32 rows are staged in shared memory by
// asynchronous copies, two stages deep, so the next stage streams in while
// the tensor cores work on the current one; at the end each warp converts its
// two exact level sums to FP64 with the scales,
// the seven warps' values are added in a fixed order, and the tile is written
// as the sub-chunk's partial.  A fixed-order sum over sub-chunks gives C.
#include "cqr_common.cuh"

namespace cqr {

namespace {

constexpr int kSub = 4096;          // rows per sub-chunk (exact FP32 level sums)
constexpr int kPlanes = 14;         // nibbles: 56 bits
constexpr int kOzWarps = 7;
constexpr int kOzThreads = 32 * kOzWarps;
constexpr int kTile = 32;           // output tile (p and q)
constexpr int kStage = 32;          // rows per shared-memory stage (one k32 MMA step)
constexpr int kLdk = kStage + 16;   // bytes per column row in shared memory (conflict-free fragments)
constexpr int kBufBytes = 2 * kPlanes * kTile * kLdk;  // one stage of both operands
constexpr int kStagesPerSub = kSub / kStage;
constexpr int kExpZero = -100000;   // scale of an all-zero column
constexpr int kExpBad = 100000;     // a column holding Inf or NaN

// e4m3 codes of 0..15 (exact): 0, 1.0, 2, 3, 4, 5, 6, 7, 8, 9, ..., 15.
__device__ __forceinline__ uint32_t e4m3_of_nibble(uint32_t n) {
  // bytes for 0..7 from two lookup words, 8..15 are 0x48 + n (linear)
  const uint32_t lo = __byte_perm(0x44403800u, 0x4E4C4A48u, n & 7u);
  return n < 8 ? (lo & 0xFFu) : (0x48u + n);
}

// ---------------------------------------------------------------------------
// Splitting: X (rows r0 .. r0 + nsub*kSub of an m x c matrix) -> planes.
// Grid (nsub, c); 256 threads; thread t handles rows 16t .. 16t+15 of the
// sub-chunk as four words of four consecutive rows.
// planes layout: byte ((s * kStagesPerSub + st) * kPlanes + i) * c * 32 +
// col * 32 + (row in stage); exps: [s * c + col].
__global__ void __launch_bounds__(256) ozaki_split_kernel(const double* X, i64 ldx, i64 m, i64 r0, int c,
                                                          uint8_t* planes, int* exps, const int* status) {
  if (status && *status) return;
  const int s = blockIdx.x, col = blockIdx.y, t = threadIdx.x;
  const i64 base = r0 + (i64)s * kSub + 16 * t;
  const double* xc = X + (i64)col * ldx;
  unsigned long long bits[16];
  int emax = -2000;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const i64 r = base + k;
    const double v = r < m ? xc[r] : 0.0;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    bits[k] = b;
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0x7FF) bad = true;
    if (E != 0 && E > emax) emax = E;  // zeros and subnormals do not set the scale
  }
  __shared__ int red_max[256 / 32];
  __shared__ int red_bad[256 / 32];
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  const int anybad = __any_sync(0xffffffffu, bad);
  if ((t & 31) == 0) {
    red_max[t >> 5] = emax;
    red_bad[t >> 5] = anybad;
  }
  __syncthreads();
  int E_max = -2000, B = 0;
  for (int w = 0; w < 256 / 32; ++w) {
    E_max = max(E_max, red_max[w]);
    B |= red_bad[w];
  }
  // |x| < 2^(E - 1022) for biased exponent E; scale e with |x| < 2^(e - 1): e = E_max - 1021
  const int e = B ? kExpBad : (E_max < 0 ? kExpZero : E_max - 1021);
  if (t == 0) exps[(i64)s * c + col] = e;
  uint32_t words[kPlanes][4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
#pragma unroll
    for (int i = 0; i < kPlanes; ++i) words[i][g] = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned long long b = bits[4 * g + k];
      const int E = (int)((b >> 52) & 0x7FF);
      unsigned long long mag = 0ull;
      if (E != 0 && E != 0x7FF && e != kExpBad) {
        const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = E - 1019 - e;  // |x| 2^(56-e) = M 2^(E - 1075 + 56 - e)
        mag = sh >= 0 ? (M << sh) : (sh > -64 ? (M >> (-sh)) : 0ull);
      }
      const uint32_t sign = (uint32_t)(b >> 63) << 7;
#pragma unroll
      for (int i = 0; i < kPlanes; ++i) {
        const uint32_t n = (uint32_t)(mag >> (4 * i)) & 15u;
        const uint32_t code = n ? (e4m3_of_nibble(n) | sign) : 0u;
        words[i][g] |= code << (8 * k);
      }
    }
  }
  const int st = (16 * t) / kStage, inrow = (16 * t) % kStage;
  uint8_t* dst = planes + ((i64)s * kStagesPerSub + st) * kPlanes * c * kStage + (i64)col * kStage + inrow;
#pragma unroll
  for (int i = 0; i < kPlanes; ++i) {
    uint4 v = make_uint4(words[i][0], words[i][1], words[i][2], words[i][3]);
    *reinterpret_cast<uint4*>(dst + (i64)i * c * kStage) = v;
  }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ void mma_e4m3(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Partial tile of C = X^T Y for one sub-chunk.  Grid (nsub, tiles_p, tiles_q).
struct OzArgs {
  const uint8_t* px;  // planes of X (p columns)
  const uint8_t* py;  // planes of Y (q columns)
  const int* ex;
  const int* ey;
  int p, q;
  int s_off;          // sub-chunk index offset of this launch in the partial buffer
  double* part;       // [s][p * q] column-major p x q
  const int* status;
};

__global__ void __launch_bounds__(kOzThreads, 2) ozaki_tn_kernel(OzArgs a) {
  extern __shared__ __align__(16) uint8_t osm[];
  if (a.status && *a.status) return;
  const int s = blockIdx.x;
  const int p0 = blockIdx.y * kTile, q0 = blockIdx.z * kTile;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int lvA = 13 + warp, lvB = 26 - warp;        // weight levels i + j of this warp
  float accA[2][4][4], accB[2][4][4];
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) accA[mi][ni][r] = accB[mi][ni][r] = 0.f;

  // Per-thread copy plan of one stage (identical for every stage up to the
  // stage base): 2 operands x 14 planes x 32 columns x 32 bytes = 1792
  // pieces of 16 bytes, 8 per thread.
  constexpr int kPieces = 2 * kPlanes * kTile * (kStage / 16);
  constexpr int kPer = kPieces / kOzThreads;
  static_assert(kPieces % kOzThreads == 0, "copy plan");
  int src_off[kPer];  // within one stage of one operand (< 14 * 1024 * 32 bytes); -1: beyond the last column
  int dst_off[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int e = t + k * kOzThreads;
    const int op = e / (kPieces / 2);
    const int r = e % (kPieces / 2);
    const int pl = r / (kTile * 2), within = r % (kTile * 2);
    const int colp = within >> 1, piece = within & 1;
    const int c = op == 0 ? a.p : a.q;
    const int colg = (op == 0 ? p0 : q0) + colp;
    src_off[k] = colg < c ? pl * c * kStage + colg * kStage + 16 * piece : -1;
    dst_off[k] = (op * kPlanes * kTile + pl * kTile + colp) * kLdk + 16 * piece;
  }
  const i64 stage_x = (i64)kPlanes * a.p * kStage, stage_y = (i64)kPlanes * a.q * kStage;
  const uint8_t* bx = a.px + (i64)s * kStagesPerSub * stage_x;
  const uint8_t* by = a.py + (i64)s * kStagesPerSub * stage_y;
  auto issue = [&](int st, uint8_t* buf) {
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int e = t + k * kOzThreads;
      const uint8_t* src = (e < kPieces / 2 ? bx + st * stage_x : by + st * stage_y) + (src_off[k] < 0 ? 0 : src_off[k]);
      cp_async16(buf + dst_off[k], src, src_off[k] < 0 ? 0 : 16);  // zero fill beyond the last column
    }
  };
  issue(0, osm);
  cp_async_commit();
  for (int st = 0; st < kStagesPerSub; ++st) {
    if (st + 1 < kStagesPerSub) issue(st + 1, osm + ((st + 1) & 1) * kBufBytes);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    const uint8_t* sx = osm + (st & 1) * kBufBytes + (16 * 0 + g) * kLdk + 4 * tq;   // + (i*kTile + 16 mi) * kLdk
    const uint8_t* sy = osm + (st & 1) * kBufBytes + (kPlanes * kTile + g) * kLdk + 4 * tq;
    // plane i of X against planes j = lvA - i and lvB - i of Y (warp-uniform predicates)
#pragma unroll
    for (int i = 0; i < kPlanes; ++i) {
      const int jA = lvA - i, jB = lvB - i;
      const bool useA = jA < kPlanes, useB = jB < kPlanes;  // j >= 0 always holds (lvA, lvB >= 13)
      if (useA || useB) {
        uint32_t af[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
          const uint8_t* base = sx + (i * kTile + 16 * mi) * kLdk;
          af[mi][0] = *reinterpret_cast<const uint32_t*>(base);
          af[mi][1] = *reinterpret_cast<const uint32_t*>(base + 8 * kLdk);
          af[mi][2] = *reinterpret_cast<const uint32_t*>(base + 16);
          af[mi][3] = *reinterpret_cast<const uint32_t*>(base + 8 * kLdk + 16);
        }
        if (useA) {
#pragma unroll
          for (int ni = 0; ni < 4; ++ni) {
            const uint8_t* bb = sy + (jA * kTile + 8 * ni) * kLdk;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(bb);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(bb + 16);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) mma_e4m3(accA[mi][ni], af[mi][0], af[mi][1], af[mi][2], af[mi][3], b0, b1);
          }
        }
        if (useB) {
#pragma unroll
          for (int ni = 0; ni < 4; ++ni) {
            const uint8_t* bb = sy + (jB * kTile + 8 * ni) * kLdk;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(bb);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(bb + 16);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) mma_e4m3(accB[mi][ni], af[mi][0], af[mi][1], af[mi][2], af[mi][3], b0, b1);
          }
        }
      }
    }
    __syncthreads();  // the buffer is refilled two stages later
  }
  // this warp's two exact level sums -> FP64 (weights 16^lv, exact powers of two)
  double* red = reinterpret_cast<double*>(osm);  // [kOzWarps][kTile * kTile]
  const double wA = ldexp(1.0, 4 * lvA), wB = ldexp(1.0, 4 * lvB);
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = 16 * mi + g + (r >= 2 ? 8 : 0);  // p index in tile
        const int col = 8 * ni + 2 * tq + (r & 1);       // q index in tile
        red[warp * kTile * kTile + row + col * kTile] = (double)accA[mi][ni][r] * wA + (double)accB[mi][ni][r] * wB;
      }
  __syncthreads();
  for (int e = t; e < kTile * kTile; e += kOzThreads) {
    const int row = e % kTile, col = e / kTile;
    const int pr = p0 + row, qc = q0 + col;
    if (pr >= a.p || qc >= a.q) continue;
    double v = 0.0;
    for (int w = 0; w < kOzWarps; ++w) v += red[w * kTile * kTile + e];
    const int ex = a.ex[(i64)s * a.p + pr], ey = a.ey[(i64)s * a.q + qc];
    double scale;
    if (ex == kExpBad || ey == kExpBad)
      scale = __longlong_as_double(0x7ff8000000000000LL);
    else if (ex == kExpZero || ey == kExpZero)
      scale = 0.0;
    else
      scale = ldexp(1.0, ex + ey - 112);
    a.part[(i64)(a.s_off + s) * a.p * a.q + pr + (i64)qc * a.p] = v * scale;
  }
}

__global__ void ozaki_reduce_kernel(const double* part, i64 nsub, int p, int q, double* C, i64 ldc,
                                    const int* status) {
  if (status && *status) return;
  const i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (i64)p * q) return;
  const int r = (int)(e % p), c = (int)(e / p);
  double s = 0.0;
  for (i64 k = 0; k < nsub; ++k) s += part[k * p * q + e];
  C[r + (i64)c * ldc] = s;
}

inline size_t oz_smem() {
  const size_t planes = (size_t)2 * kBufBytes;
  const size_t red = sizeof(double) * kOzWarps * kTile * kTile;
  return planes > red ? planes : red;
}

}  // namespace

// Rows per splitting chunk: planes of one chunk take about 1 GiB.
i64 oz_chunk_rows(int p, int q) {
  i64 rows = ((i64)1 << 30) / ((i64)kPlanes * (p + q));
  rows = (rows / kSub) * kSub;
  return rows < kSub ? kSub : rows;
}

size_t ozaki_workspace_bytes(i64 m, int p, int q) {
  if (m <= 0 || p <= 0 || q <= 0) return 0;
  const i64 nsub_total = (m + kSub - 1) / kSub;
  i64 ch = oz_chunk_rows(p, q);
  const i64 mr = ((m + kSub - 1) / kSub) * kSub;
  if (ch > mr) ch = mr;
  const i64 nsub_ch = ch / kSub;
  size_t b = 0;
  b += (size_t)nsub_ch * kPlanes * (p + q) * kSub;           // planes of one chunk
  b = (b + 255) & ~(size_t)255;
  b += sizeof(int) * (size_t)nsub_ch * (p + q);               // scales
  b = (b + 255) & ~(size_t)255;
  b += sizeof(double) * (size_t)nsub_total * p * q;           // partials
  return (b + 255) & ~(size_t)255;
}

cudaError_t tn_product_emulated(i64 m, int p, int q, const double* X, i64 ldx, const double* Y, i64 ldy,
                                void* ws, double* C, i64 ldc, const int* status, cudaStream_t st) {
  if (p <= 0 || q <= 0) return cudaSuccess;
  const i64 nsub_total = (m + kSub - 1) / kSub;
  i64 ch = oz_chunk_rows(p, q);
  const i64 mr = nsub_total * kSub;
  if (ch > mr) ch = mr;
  const i64 nsub_ch = ch / kSub;
  uint8_t* planes = (uint8_t*)ws;
  size_t off = (size_t)nsub_ch * kPlanes * (p + q) * kSub;
  off = (off + 255) & ~(size_t)255;
  int* exps = (int*)((char*)ws + off);
  off += sizeof(int) * (size_t)nsub_ch * (p + q);
  off = (off + 255) & ~(size_t)255;
  double* part = (double*)((char*)ws + off);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(ozaki_tn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem());
    attr = true;
  }
  uint8_t* px = planes;
  uint8_t* py = planes + (size_t)nsub_ch * kPlanes * p * kSub;
  int* ex = exps;
  int* ey = exps + nsub_ch * p;
  for (i64 r0 = 0; r0 < m; r0 += ch) {
    const i64 nsub = ((m - r0 < ch ? m - r0 : ch) + kSub - 1) / kSub;
    prof_begin(kMisc, st);
    ozaki_split_kernel<<<dim3((unsigned)nsub, (unsigned)p), 256, 0, st>>>(X, ldx, m, r0, p, px, ex, status);
    prof_end(kMisc, 0.0, st);
    prof_begin(kMisc, st);
    ozaki_split_kernel<<<dim3((unsigned)nsub, (unsigned)q), 256, 0, st>>>(Y, ldy, m, r0, q, py, ey, status);
    prof_end(kMisc, 0.0, st);
    OzArgs a;
    a.px = px;
    a.py = py;
    a.ex = ex;
    a.ey = ey;
    a.p = p;
    a.q = q;
    a.s_off = (int)(r0 / kSub);
    a.part = part;
    a.status = status;
    dim3 grid((unsigned)nsub, (unsigned)((p + kTile - 1) / kTile), (unsigned)((q + kTile - 1) / kTile));
    prof_begin(kProjection, st);
    ozaki_tn_kernel<<<grid, kOzThreads, oz_smem(), st>>>(a);
    prof_end(kProjection, 2.0 * (double)(nsub * kSub < m - r0 ? nsub * kSub : m - r0) * p * q, st);
  }
  const i64 pq = (i64)p * q;
  prof_begin(kReduce, st);
  ozaki_reduce_kernel<<<(unsigned)((pq + 255) / 256), 256, 0, st>>>(part, nsub_total, p, q, C, ldc, status);
  prof_end(kReduce, (double)nsub_total * pq, st);
  return cudaGetLastError();
}

}  // namespace cqr
