// FP64-accurate split-m products on the FP8 tensor cores (the Ozaki
// error-free splitting; Ozaki, Ogita, Oishi, Numer. Algorithms 59 (2012)),
// for the emulated variant of Alg. 9 (opt-in, CQR_EMULATED): the projections
// C = X^T Y of steps 3 and 7 and the updates C -= X Y of steps 4 and 7.
//
// Splitting.  For C = X^T Y, rows are cut into sub-chunks of kSub = 4096.
// Within a sub-chunk every column c of X (and of Y) gets a power-of-two
// scale 2^e_c with |x| < 2^e_c, and each entry becomes the 56-bit
// fixed-point integer |x| * 2^(56 - e_c) (truncated below 2^-56 of the scale)
// split into 14 unsigned nibbles n_0..n_13 (n_i has weight 16^i); digit i of
// x is sign(x) * n_i, an integer in [-15, 15] that e4m3 represents exactly.
// Digits live in 14 "planes" laid out [sub-chunk][32-row stage][plane]
// [column][32 bytes], so that one stage of a 32-column tile is 14
// contiguous 1 KiB runs per operand.  For C -= X Y the contraction runs over
// the columns of X: each row of X gets its own scale over (at most kSub of)
// its entries and its digits take the place of a column in the same layout;
// Y (K x N) is split by columns as before.
//
// Products.  x_a y_b = 2^(e_a + e_b - 112) sum_{i,j} d^x_i d^y_j 16^(i+j).
// The plane pairs with i + j >= kLevelLo (the 27 - kLevelLo most significant
// weight levels) are multiplied with mma.sync m16n8k32 e4m3 -> f32.  Per
// level the sum over at most 4096 contraction indices is below
// 14 * 225 * 4096 < 2^24 in magnitude, so the FP32 accumulation is exact (an
// integer).  With kLevelLo = 13 (105 pairs) the dropped levels weigh at most
// about 2^-52.5 of the scales' product per index, so below 2^-50.5 of the
// product of the two largest magnitudes.
//
// Schedule.  A block ((27 - kLevelLo) / 2 warps) computes a 32 x 32 tile of
// C: warp w owns levels kLevelLo + w and 26 - w (for kLevelLo = 13: 15 plane
// pairs, equal for every warp); the
// planes of 32 contraction indices are staged in shared memory by
// asynchronous copies, two stages deep, so the next stage streams in while
// the tensor cores work on the current one.  At the end the 14 exact level
// sums of every element go through shared memory as integers; groups of
// seven levels are each combined exactly in 64-bit integers (below 2^49) and
// joined by FP64 fused multiply-adds (one rounding for two groups), so the
// FP64 pipe does a handful of operations per element.
// A projection tile is a sub-chunk's partial (a fixed-order sum over
// sub-chunks gives C); an update tile is subtracted from C.
#include "cqr_common.cuh"

namespace cqr {

namespace {

constexpr int kSub = 4096;          // rows per sub-chunk (exact FP32 level sums)
constexpr int kPlanes = 14;         // nibbles: 56 bits
constexpr int kLevelLo = 13;        // lowest weight level i + j kept
constexpr int kLevels = 2 * kPlanes - 1 - kLevelLo;
static_assert(kLevels % 2 == 0 && kLevels <= 21, "two levels per warp, at most three groups of seven");
constexpr int kOzWarps = kLevels / 2;
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

// Digits of one FP64 value (raw bits b) against scale e into byte k of
// word g of the 14 plane words.
__device__ __forceinline__ void put_digits(unsigned long long b, int e, uint32_t (&words)[kPlanes][4], int g, int k) {
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
  // |x| < 2^(E - 1022) for biased exponent E; scale e with |x| < 2^e: e = E_max - 1022
  const int e = B ? kExpBad : (E_max < 0 ? kExpZero : E_max - 1022);
  if (t == 0) exps[(i64)s * c + col] = e;
  uint32_t words[kPlanes][4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
#pragma unroll
    for (int i = 0; i < kPlanes; ++i) words[i][g] = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) put_digits(bits[4 * g + k], e, words, g, k);
  }
  const int st = (16 * t) / kStage, inrow = (16 * t) % kStage;
  uint8_t* dst = planes + ((i64)s * kStagesPerSub + st) * kPlanes * c * kStage + (i64)col * kStage + inrow;
#pragma unroll
  for (int i = 0; i < kPlanes; ++i) {
    uint4 v = make_uint4(words[i][0], words[i][1], words[i][2], words[i][3]);
    *reinterpret_cast<uint4*>(dst + (i64)i * c * kStage) = v;
  }
}

// Row splitting for C -= X Y: rows r0 .. r0 + rows of X (m x K, ldx) over the
// contraction columns k0 .. k0 + kc (kc <= kSub).  Thread = row; every row
// gets its own scale over its kc entries (first pass), then its digits for
// 16 columns at a time (second pass) go to byte ((st * kPlanes + i) * rows +
// row) * 32 + (k - k0) % 32 with st = (k - k0) / 32: the column layout above
// with rows in the role of columns.  rows is a multiple of 32; rows at or
// past m split as zeros.
__global__ void __launch_bounds__(128) ozaki_rowsplit_kernel(const double* X, i64 ldx, i64 m, i64 r0, int rows,
                                                             i64 k0, int kc, uint8_t* planes, int* exps,
                                                             const int* status) {
  if (status && *status) return;
  const int row = blockIdx.x * 128 + threadIdx.x;
  if (row >= rows) return;
  const i64 r = r0 + row;
  const bool live = r < m;
  const double* xr = X + (live ? r : 0) + k0 * ldx;
  int emax = -2000;
  bool bad = false;
  if (live) {
#pragma unroll 8
    for (int k = 0; k < kc; ++k) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(xr[(i64)k * ldx]);
      const int E = (int)((b >> 52) & 0x7FF);
      bad |= E == 0x7FF;
      if (E != 0 && E > emax) emax = E;
    }
  }
  const int e = bad ? kExpBad : (emax < 0 ? kExpZero : emax - 1022);
  exps[row] = e;
  const int nst = (kc + kStage - 1) / kStage;
  for (int st = 0; st < nst; ++st) {
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int kb = st * kStage + 16 * h;
      uint32_t words[kPlanes][4];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
#pragma unroll
        for (int i = 0; i < kPlanes; ++i) words[i][g] = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int kk = kb + 4 * g + k;
          const double v = (live && kk < kc) ? xr[(i64)kk * ldx] : 0.0;
          put_digits((unsigned long long)__double_as_longlong(v), e, words, g, k);
        }
      }
      uint8_t* dst = planes + ((i64)st * kPlanes * rows + row) * kStage + 16 * h;
#pragma unroll
      for (int i = 0; i < kPlanes; ++i) {
        uint4 v = make_uint4(words[i][0], words[i][1], words[i][2], words[i][3]);
        *reinterpret_cast<uint4*>(dst + (i64)i * rows * kStage) = v;
      }
    }
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
// One 32 x 32 tile of C.  Projection (NN = false): grid (nsub, tiles_p,
// tiles_q), the tile of sub-chunk s goes to the partial buffer.  Update
// (NN = true): one launch per chunk of rows, a linear grid with the q tile
// fastest (the blocks of one row tile run together and share its X planes
// in L2), and C -= tile.
struct OzArgs {
  const uint8_t* px;  // planes of X (projection: p columns; update: p rows)
  const uint8_t* py;  // planes of Y (q columns)
  const int* ex;
  const int* ey;
  int p, q;
  int s_off;          // projection: sub-chunk index offset of this launch in the partial buffer
  double* part;       // projection: [s][p * q] column-major p x q
  int nst;            // update: stages of 32 contraction indices
  int tiles_q;        // update: ceil(q / 32)
  int p_live;         // update: rows of the chunk that exist (p rounded up to 32 is the planes' row count)
  double* C;          // update: C (ldc) of the chunk's first row
  i64 ldc;
  const int* status;
};

constexpr int kLvlLd = kTile + 4;  // level-sum staging: column stride in ints (conflict-free writes)

template <bool NN>
__global__ void __launch_bounds__(kOzThreads, 2) ozaki_kernel(OzArgs a) {
  extern __shared__ __align__(16) uint8_t osm[];
  if (a.status && *a.status) return;
  int s, p0, q0, nst;
  if (NN) {
    s = 0;
    q0 = (int)(blockIdx.x % (unsigned)a.tiles_q) * kTile;
    p0 = (int)(blockIdx.x / (unsigned)a.tiles_q) * kTile;
    nst = a.nst;
  } else {
    s = blockIdx.x;
    p0 = blockIdx.y * kTile;
    q0 = blockIdx.z * kTile;
    nst = kStagesPerSub;
  }
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int lvA = kLevelLo + warp, lvB = 2 * kPlanes - 2 - warp;  // weight levels i + j of this warp
  float accA[2][4][4], accB[2][4][4];
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) accA[mi][ni][r] = accB[mi][ni][r] = 0.f;

  // Copy plan of one stage: 2 operands x 14 planes x 32 columns x 32 bytes =
  // 1792 pieces of 16 bytes, the same number per thread; the offsets are
  // recomputed per stage, which costs a few integer operations and keeps the
  // registers for the accumulators.
  constexpr int kPieces = 2 * kPlanes * kTile * (kStage / 16);
  constexpr int kPer = kPieces / kOzThreads;
  static_assert(kPieces % kOzThreads == 0, "copy plan");
  const i64 stage_x = (i64)kPlanes * a.p * kStage, stage_y = (i64)kPlanes * a.q * kStage;
  const uint8_t* bx = a.px + (i64)s * kStagesPerSub * stage_x;
  const uint8_t* by = a.py + (i64)s * kStagesPerSub * stage_y;
  auto issue = [&](int st, uint8_t* buf) {
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int e = t + kOzThreads * k;
      const int op = e >= kPieces / 2 ? 1 : 0;
      const int r = e - op * (kPieces / 2);
      const int pl = r / (kTile * 2), within = r % (kTile * 2);
      const int colp = within >> 1, piece = within & 1;
      const int c = op == 0 ? a.p : a.q;
      const int colg = (op == 0 ? p0 : q0) + colp;
      const bool ok = colg < c;  // zero fill beyond the last column; offsets < 14 * c * 32 < 2^31
      const uint8_t* src = (op == 0 ? bx + st * stage_x : by + st * stage_y) +
                           (ok ? pl * c * kStage + colg * kStage + 16 * piece : 0);
      cp_async16(buf + (op * kPlanes * kTile + pl * kTile + colp) * kLdk + 16 * piece, src, ok ? 16 : 0);
    }
  };
  issue(0, osm);
  cp_async_commit();
  for (int st = 0; st < nst; ++st) {
    if (st + 1 < nst) issue(st + 1, osm + ((st + 1) & 1) * kBufBytes);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    const uint8_t* sx = osm + (st & 1) * kBufBytes + (16 * 0 + g) * kLdk + 4 * tq;   // + (i*kTile + 16 mi) * kLdk
    const uint8_t* sy = osm + (st & 1) * kBufBytes + (kPlanes * kTile + g) * kLdk + 4 * tq;
    // plane i of X against planes j = lvA - i and lvB - i of Y (warp-uniform predicates)
#pragma unroll
    for (int i = 0; i < kPlanes; ++i) {
      const int jA = lvA - i, jB = lvB - i;
      const bool useA = jA >= 0 && jA < kPlanes, useB = jB >= 0 && jB < kPlanes;
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
  // the level sums are exact integers below 2^24: stage them as int32,
  // [level - 13][col * kLvlLd + row]
  int* lvl = reinterpret_cast<int*>(osm);
  constexpr int kLvlStride = kTile * kLvlLd;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = 16 * mi + g + (r >= 2 ? 8 : 0);  // p index in tile
        const int col = 8 * ni + 2 * tq + (r & 1);       // q index in tile
        lvl[(lvA - kLevelLo) * kLvlStride + col * kLvlLd + row] = __float2int_rz(accA[mi][ni][r]);
        lvl[(lvB - kLevelLo) * kLvlStride + col * kLvlLd + row] = __float2int_rz(accB[mi][ni][r]);
      }
  __syncthreads();
  const int p_end = NN ? a.p_live : a.p;
  for (int e = t; e < kTile * kTile; e += kOzThreads) {
    const int row = e % kTile, col = e / kTile;
    const int pr = p0 + row, qc = q0 + col;
    if (pr >= p_end || qc >= a.q) continue;
    // sum_L S_L 16^L = 16^kLevelLo (g0 + 2^28 g1 + 2^56 g2), group g_i = sum of
    // S_L 16^(L - kLevelLo - 7 i) over its (at most seven) levels
    const int* le = lvl + col * kLvlLd + row;
    long long grp[3] = {0, 0, 0};
#pragma unroll
    for (int L = kLevels - 1; L >= 0; --L) grp[L / 7] = grp[L / 7] * 16 + le[L * kLvlStride];
    // |g_i| < 2^49: exact operands; one rounding per fused multiply-add
    const double v = fma((double)grp[2], 72057594037927936.0, fma((double)grp[1], 268435456.0, (double)grp[0]));
    const int ex = a.ex[(i64)s * a.p + pr], ey = a.ey[(i64)s * a.q + qc];
    double scale;
    if (ex == kExpBad || ey == kExpBad)
      scale = __longlong_as_double(0x7ff8000000000000LL);
    else if (ex == kExpZero || ey == kExpZero)
      scale = 0.0;
    else
      scale = ldexp(1.0, ex + ey - 112 + 4 * kLevelLo);
    if (NN) {
      double* cp = a.C + pr + (i64)qc * a.ldc;
      *cp -= v * scale;
    } else {
      a.part[(i64)(a.s_off + s) * a.p * a.q + pr + (i64)qc * a.p] = v * scale;
    }
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
  const size_t lv = sizeof(int) * kLevels * kTile * kLvlLd;
  return planes > lv ? planes : lv;
}

// Rows per update chunk: the X planes of one chunk take about 1 GiB.
inline i64 oz_nn_rows(int nst) {
  i64 rows = ((i64)1 << 30) / ((i64)kPlanes * kStage * nst);
  rows = rows / kTile * kTile;
  return rows < kTile ? kTile : rows;
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
    cudaFuncSetAttribute(ozaki_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem());
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
    OzArgs a{};
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
    ozaki_kernel<false><<<grid, kOzThreads, oz_smem(), st>>>(a);
    prof_end(kProjection, 2.0 * (double)(nsub * kSub < m - r0 ? nsub * kSub : m - r0) * p * q, st);
  }
  const i64 pq = (i64)p * q;
  prof_begin(kReduce, st);
  ozaki_reduce_kernel<<<(unsigned)((pq + 255) / 256), 256, 0, st>>>(part, nsub_total, p, q, C, ldc, status);
  prof_end(kReduce, (double)nsub_total * pq, st);
  return cudaGetLastError();
}

size_t ozaki_nn_workspace_bytes(i64 M, int N, int K) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  const int kc = K < kSub ? K : kSub;
  const int nst = (kc + kStage - 1) / kStage;
  i64 rows = oz_nn_rows(nst);
  const i64 mr = (M + kTile - 1) / kTile * kTile;
  if (rows > mr) rows = mr;
  size_t b = (size_t)rows * nst * kStage * kPlanes;  // X planes of one chunk
  b = (b + 255) & ~(size_t)255;
  b += (size_t)kSub * kPlanes * N;                   // Y planes (one sub-chunk)
  b = (b + 255) & ~(size_t)255;
  b += sizeof(int) * ((size_t)rows + N);             // scales
  return (b + 255) & ~(size_t)255;
}

cudaError_t nn_update_emulated(i64 M, int N, int K, const double* X, i64 ldx, const double* Y, i64 ldy, double* C,
                               i64 ldc, void* ws, const int* status, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  const int kcmax = K < kSub ? K : kSub;
  const int nstmax = (kcmax + kStage - 1) / kStage;
  i64 rows = oz_nn_rows(nstmax);
  const i64 mr = (M + kTile - 1) / kTile * kTile;
  if (rows > mr) rows = mr;
  uint8_t* px = (uint8_t*)ws;
  size_t off = ((size_t)rows * nstmax * kStage * kPlanes + 255) & ~(size_t)255;
  uint8_t* py = (uint8_t*)ws + off;
  off = (off + (size_t)kSub * kPlanes * N + 255) & ~(size_t)255;
  int* ex = (int*)((char*)ws + off);
  int* ey = ex + rows;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(ozaki_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem());
    attr = true;
  }
  const int tiles_q = (N + kTile - 1) / kTile;
  for (i64 k0 = 0; k0 < K; k0 += kSub) {
    const int kc = (int)(K - k0 < kSub ? K - k0 : kSub);
    const int nst = (kc + kStage - 1) / kStage;
    prof_begin(kMisc, st);
    ozaki_split_kernel<<<dim3(1u, (unsigned)N), 256, 0, st>>>(Y, ldy, k0 + kc, k0, N, py, ey, status);
    prof_end(kMisc, 0.0, st);
    for (i64 r0 = 0; r0 < M; r0 += rows) {
      const i64 live = M - r0 < rows ? M - r0 : rows;
      const int rws = (int)((live + kTile - 1) / kTile * kTile);
      prof_begin(kMisc, st);
      ozaki_rowsplit_kernel<<<(unsigned)((rws + 127) / 128), 128, 0, st>>>(X, ldx, M, r0, rws, k0, kc, px, ex,
                                                                          status);
      prof_end(kMisc, 0.0, st);
      OzArgs a{};
      a.px = px;
      a.py = py;
      a.ex = ex;
      a.ey = ey;
      a.p = rws;
      a.q = N;
      a.nst = nst;
      a.tiles_q = tiles_q;
      a.p_live = (int)live;
      a.C = C + r0;
      a.ldc = ldc;
      a.status = status;
      prof_begin(kUpdate, st);
      ozaki_kernel<true><<<(unsigned)((i64)(rws / kTile) * tiles_q), kOzThreads, oz_smem(), st>>>(a);
      prof_end(kUpdate, 2.0 * (double)live * N * kc, st);
    }
  }
  return cudaGetLastError();
}

}  // namespace cqr
