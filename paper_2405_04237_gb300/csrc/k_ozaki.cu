// FP64-accurate split-m products on the 5th-generation (tcgen05) FP8 tensor
// cores, with the Ozaki error-free splitting (Ozaki, Ogita, Oishi, Numer.
// Algorithms 59 (2012)), for the emulated variant of Alg. 9 (opt-in,
// CQR_EMULATED): the projections C = X^T Y of steps 3 and 7 and the updates
// C -= X Y of steps 4 and 7.
//
// Splitting.  For C = X^T Y, rows are cut into sub-chunks of kSub = 4096.
// Within a sub-chunk every column c of X (and of Y) gets a power-of-two
// scale 2^e_c with |x| < 2^e_c, and each entry becomes the 56-bit fixed-point
// integer |x| * 2^(56 - e_c) (truncated below 2^-56 of the scale) split into
// 14 unsigned nibbles n_0..n_13 (n_i has weight 16^i); digit i of x is
// sign(x) * n_i, an integer in [-15, 15] that e4m3 represents exactly.  For
// C -= X Y the contraction runs over the columns of X: each row of X gets its
// own scale over (at most kSub of) its entries and takes a column's place;
// Y (K x N) is split by columns.
//
// Plane layout.  One "stage" is 32 contraction indices.  Columns are grouped
// in tiles of T (128 on the X side, 32 on the Y side), and the planes are
// stored tile-major: for each tile, each stage, each plane i, the T x 32
// digits in the tensor cores' canonical K-major layout without swizzling
// (8-column groups of 256 bytes, each two 8 x 16-byte core matrices holding
// indices 0..15, then 16..31).  The 14 planes of one stage of one tile are
// thus one contiguous run (56 KiB for X, 14 KiB for Y), and a stage arrives
// in shared memory with two bulk asynchronous copies (for a Gram matrix
// X^T X, whose Y tiles are 32-column slices of the X planes, one copy for X
// and one per plane for Y).
//
// Products.  x_a y_b = 2^(e_a + e_b - 112) sum_{i,j} d^x_i d^y_j 16^(i+j).
// The 105 plane pairs with i + j >= 13 (the 14 most significant weight
// levels) are multiplied with tcgen05.mma kind::f8f6f4 (e4m3 x e4m3 -> f32)
// into one TMEM accumulator per level: TMEM region r (32 columns, r = 0..15)
// holds level r + 11.  The Y planes of one stage lie in shared memory one
// after the other, so planes j0 .. j0+n-1 form one operand of N = 32 n rows,
// and one instruction A_i x [Y_j0; ...; Y_j0+n-1] (128 x 32n x 32) adds pair
// (i, j0 + v) into region i + j0 + v - 11 for v < n.  22 such instructions
// (N = 32 .. 256) cover the 105 pairs, plus 6 pairs of levels 11 and 12,
// whose regions are never read.  Per level the sum over at most 4096
// contraction indices is below 14 * 225 * 4096 < 2^24 in magnitude, so the
// FP32 accumulation is exact (an integer).  The dropped levels weigh at most
// about 2^-52.5 of the scales' product per index, so below 2^-50.5 of the
// product of the two largest magnitudes.
//
// Schedule.  A block of 4 warps computes a 128 x 32 tile of C over its
// contraction range (a sub-chunk of a projection, all of K for an update).
// Three shared-memory stages of 70 KiB rotate: one thread issues the bulk
// copies of a stage (completion counted in bytes on the stage's "full"
// mbarrier), one thread issues its 22 MMAs and commits them to the stage's
// "empty" mbarrier, which frees the stage for the copy three stages later.
// At the end every thread reads the 14 level sums of its row from TMEM,
// combines levels 13..19 and 20..26 exactly in 64-bit integers (below 2^49),
// builds the two scaled doubles with integer operations and adds them (one
// rounding), so the FP64 pipe does one operation per element (two for an
// update, which subtracts the tile from C).  Every wait is bounded in time
// (kWaitNs of the global nanosecond timer, 2 s: a stage arrives within
// microseconds); on expiry the block records CQR_STATUS_TIMEOUT, waits
// (bounded) for its copies in flight, frees its TMEM and returns.  A
// one-shot host-side test hook (cqr_test_arm_wait_expiry) makes the next
// launch of one of the two kernels withhold the copies of one stage, with a
// short bound, so that the expiry path runs and can be checked.
#include <mutex>

#include "cqr_common.cuh"
#include "cqr.h"

namespace cqr {

namespace {

constexpr int kSub = 4096;          // rows per sub-chunk (exact FP32 level sums)
constexpr int kPlanes = 14;         // nibbles: 56 bits
constexpr int kLevelLo = 13;        // lowest weight level i + j kept
constexpr int kLevels = 2 * kPlanes - 1 - kLevelLo;
constexpr int kStage = 32;          // contraction indices per stage (one MMA K step for 8-bit types)
constexpr int kStagesPerSub = kSub / kStage;
constexpr int kExpZero = -100000;   // scale of an all-zero column
constexpr int kExpBad = 100000;     // a column holding Inf or NaN

constexpr int kTcM = 128;           // rows of the tile (X side, TMEM lanes)
constexpr int kTcN = 32;            // columns of the tile (Y side)
constexpr int kTcThreads = 128;
constexpr int kTcRing = 3;
constexpr int kTcABytes = kPlanes * kTcM * kStage;    // 57344
constexpr int kTcBBytes = kPlanes * kTcN * kStage;    // 14336
constexpr int kTcStageBytes = kTcABytes + kTcBBytes;  // 71680
constexpr int kTcSmem = kTcRing * kTcStageBytes + 1024;  // + alignment slack
constexpr uint32_t kTcCols = 512;   // TMEM columns: 16 regions of kTcN, levels 11..26
constexpr int kMaxDynSmem = 227 * 1024 - 1024;  // opt-in dynamic shared memory per block, less static use
static_assert(kTcSmem <= kMaxDynSmem, "projection ring fits in shared memory");
static_assert(kTcCols >= 32 && kTcCols <= 512 && (kTcCols & (kTcCols - 1)) == 0, "TMEM allocation: power of 2, 32..512");
constexpr int kRegionLo = 11;       // level of TMEM region 0
static_assert((2 * kPlanes - 1 - kRegionLo) * kTcN == (int)kTcCols, "level regions fill the TMEM allocation");
static_assert(kLevelLo == 13 && kLevels == 14, "the MMA schedule and the two groups of seven levels");
// Instruction descriptor of tcgen05.mma kind::f8f6f4 without N: D f32 (bits
// 4-5 = 1), A and B e4m3 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 =
// 0), M >> 4 at bits 24-28; N >> 3 goes to bits 17-22.
constexpr uint32_t kTcIdescM = (1u << 4) | ((uint32_t)(kTcM >> 4) << 24);
constexpr unsigned long long kWaitNs = 2000000000ull;  // bound of every mbarrier wait (ns of %globaltimer)

inline int round_up(int x, int t) { return (x + t - 1) / t * t; }

// 56-bit magnitude |x| * 2^(56 - e) (truncated) of one FP64 value (raw bits b)
// against scale e; zero for zeros, subnormals and a bad column.
__device__ __forceinline__ unsigned long long magnitude(unsigned long long b, int e) {
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0 || E == 0x7FF || e == kExpBad) return 0ull;
  const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = E - 1019 - e;  // |x| 2^(56-e) = M 2^(E - 1075 + 56 - e)
  return sh >= 0 ? (M << sh) : (sh > -64 ? (M >> (-sh)) : 0ull);
}

// e4m3 codes of four nibbles (one per byte of n, each 0..15): 0, 1, ..., 7
// come from two lookup words, 8..15 (0x50 + n - 8) from two more, chosen per
// byte by bit 3 of the nibble.
__device__ __forceinline__ uint32_t e4m3_of_nibbles(uint32_t n) {
  const uint32_t v = n & 0x07070707u;
  const uint32_t u = v | (v >> 4);
  const uint32_t sel = __byte_perm(u, 0u, 0x4420);  // selector nibbles v0, v1, v2, v3
  const uint32_t lo = __byte_perm(0x44403800u, 0x4E4C4A48u, sel);
  const uint32_t hi = __byte_perm(0x53525150u, 0x57565554u, sel);
  const uint32_t mask = ((n >> 3) & 0x01010101u) * 0xFFu;
  return (lo & ~mask) | (hi & mask);
}

// Digits of four FP64 values (raw bits b[0..3]) against scale e: byte k of
// word i is the e4m3 code of digit i of value k, sign(x_k) * nibble i.  The
// four 56-bit magnitudes are transposed bytewise with byte permutes, so that
// every step below works on four values at once.
__device__ __forceinline__ void digits4(const unsigned long long (&b)[4], int e, uint32_t (&w)[kPlanes]) {
  uint32_t lo[4], hi[4], sgn = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned long long m = magnitude(b[k], e);
    lo[k] = (uint32_t)m;
    hi[k] = (uint32_t)(m >> 32);
    sgn |= (uint32_t)(b[k] >> 63) << (8 * k + 7);
  }
#pragma unroll
  for (int j = 0; j < kPlanes / 2; ++j) {  // byte j of the four magnitudes
    const uint32_t* src = j < 4 ? lo : hi;
    const uint32_t sel = (uint32_t)(j & 3) | ((uint32_t)((j & 3) + 4) << 4);
    const uint32_t t01 = __byte_perm(src[0], src[1], sel);
    const uint32_t t23 = __byte_perm(src[2], src[3], sel);
    const uint32_t bj = __byte_perm(t01, t23, 0x5410);
    w[2 * j] = e4m3_of_nibbles(bj & 0x0F0F0F0Fu) | sgn;
    w[2 * j + 1] = e4m3_of_nibbles((bj >> 4) & 0x0F0F0F0Fu) | sgn;
  }
}

// Byte offset, within one (stage, plane) block, of the 16 indices
// 16*half .. 16*half+15 of column col (canonical K-major layout).
__device__ __forceinline__ i64 plane_off(i64 col, int half) {
  return (col >> 3) * 256 + half * 128 + (col & 7) * 16;
}

// ---------------------------------------------------------------------------
// Column splitting: X (rows r0 .. r0 + nsub*kSub of an m x c matrix) ->
// planes.  Grid (ceil(c / 8), nsub), 256 threads: block (g, s) takes the
// 8-column group g of the layout (columns 8g .. 8g+7) over sub-chunk s, so
// that for each stage and plane its digits form one contiguous 256-byte run
// (8 columns x 32 indices).  Lane l of warp w handles column 8g + (l & 7),
// half (l >> 3) & 1 (indices 0..15 or 16..31 of a stage) of stages
// 16 it + 2 w + (l >> 4), it = 0..7: every warp store writes two whole
// 256-byte runs.  Two passes over the sub-chunk: the column maxima (scales),
// then the digits; the second pass re-reads from L2 (at most two blocks, 2 x
// 256 KiB, per SM).  Tiles of T columns (T a multiple of 8); plane block
// (s, tile, st, i) starts at byte
// (((s * ntile + tile) * kStagesPerSub + st) * kPlanes + i) * T * 32 with
// ntile = ceil(c / T); exps: [s * c + col].  Columns past c of the last
// group are written as zero digits (the tile padding; never read).
// 16 consecutive entries xc[row .. row+15] (zero past m or for a column past
// c); 16-byte loads when the address allows (an odd leading dimension puts
// every other column off the 16-byte grid).
__device__ __forceinline__ void load16(const double* xc, i64 row, i64 m, bool colok, unsigned long long (&bits)[16]) {
  if (colok && row + 15 < m && ((reinterpret_cast<uintptr_t>(xc + row) & 15) == 0)) {
    const double2* p = reinterpret_cast<const double2*>(xc + row);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double2 v = __ldg(p + k);
      bits[2 * k] = (unsigned long long)__double_as_longlong(v.x);
      bits[2 * k + 1] = (unsigned long long)__double_as_longlong(v.y);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 16; ++k)
      bits[k] = (unsigned long long)__double_as_longlong((colok && row + k < m) ? xc[row + k] : 0.0);
  }
}

__global__ void __launch_bounds__(256, 2) ozaki_split_kernel(const double* X, i64 ldx, i64 m, i64 r0, int c, int T,
                                                             uint8_t* planes, int* exps, const int* status) {
  if (status && *status) return;
  const int g = blockIdx.x, s = blockIdx.y, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int cl = lane & 7, half = (lane >> 3) & 1, so = lane >> 4;
  const int col = 8 * g + cl;
  const bool colok = col < c;
  const i64 base = r0 + (i64)s * kSub;
  const double* xc = X + (i64)(colok ? col : 0) * ldx;
  // pass 1: the column's largest exponent (zeros and subnormals do not set the scale) and Inf/NaN
  int emax = -2000;
  bool bad = false;
#pragma unroll 1
  for (int it = 0; it < 8; ++it) {
    const int st = 16 * it + 2 * warp + so;
    unsigned long long bits[16];
    load16(xc, base + st * kStage + 16 * half, m, colok, bits);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int E = (int)((bits[k] >> 52) & 0x7FF);
      if (E == 0x7FF) bad = true;
      if (E != 0 && E > emax) emax = E;
    }
  }
  // lanes l, l ^ 8, l ^ 16, l ^ 24 hold the same column
  emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 8));
  emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 16));
  int anyb = bad ? 1 : 0;
  anyb |= __shfl_xor_sync(0xffffffffu, anyb, 8);
  anyb |= __shfl_xor_sync(0xffffffffu, anyb, 16);
  __shared__ int red_max[8][8], red_bad[8][8];
  __shared__ int e_col[8];
  if (lane < 8) {
    red_max[warp][lane] = emax;
    red_bad[warp][lane] = anyb;
  }
  __syncthreads();
  if (t < 8) {
    int E_max = -2000, B = 0;
    for (int w = 0; w < 8; ++w) {
      E_max = max(E_max, red_max[w][t]);
      B |= red_bad[w][t];
    }
    // |x| < 2^(E - 1022) for biased exponent E; scale e with |x| < 2^e: e = E_max - 1022
    const int e = B ? kExpBad : (E_max < 0 ? kExpZero : E_max - 1022);
    e_col[t] = e;
    if (8 * g + t < c) exps[(i64)s * c + 8 * g + t] = e;
  }
  __syncthreads();
  const int e = e_col[cl];
  // pass 2: digits, one 16-byte granule per plane
  const int ntile = (c + T - 1) / T;
  uint8_t* dst0 = planes + ((i64)s * ntile + col / T) * kStagesPerSub * kPlanes * T * kStage + plane_off(col % T, half);
#pragma unroll 1
  for (int it = 0; it < 8; ++it) {
    const int st = 16 * it + 2 * warp + so;
    unsigned long long bits[16];
    load16(xc, base + st * kStage + 16 * half, m, colok, bits);
    uint32_t words[kPlanes][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const unsigned long long b4[4] = {bits[4 * q], bits[4 * q + 1], bits[4 * q + 2], bits[4 * q + 3]};
      uint32_t w[kPlanes];
      digits4(b4, e, w);
#pragma unroll
      for (int i = 0; i < kPlanes; ++i) words[i][q] = w[i];
    }
    uint8_t* dst = dst0 + (i64)st * kPlanes * T * kStage;
#pragma unroll
    for (int i = 0; i < kPlanes; ++i) {
      uint4 v = make_uint4(words[i][0], words[i][1], words[i][2], words[i][3]);
      *reinterpret_cast<uint4*>(dst + (i64)i * T * kStage) = v;
    }
  }
}

// Row splitting for C -= X Y: rows r0 .. r0 + rows of X (m x K, ldx) over the
// contraction columns k0 .. k0 + kc (kc <= kSub).  Thread = row; every row
// gets its own scale over its kc entries (first pass), then its digits for
// 16 columns at a time (second pass) go to plane block (tile, st, i) at
// byte ((tile * nst + st) * kPlanes + i) * 128 * 32 with tile = row / 128,
// rows in the role of columns.  rows is a multiple of 128; rows at or past m
// split as zeros.
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
        unsigned long long b4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int kk = kb + 4 * g + k;
          b4[k] = (unsigned long long)__double_as_longlong((live && kk < kc) ? xr[(i64)kk * ldx] : 0.0);
        }
        uint32_t w[kPlanes];
        digits4(b4, e, w);
#pragma unroll
        for (int i = 0; i < kPlanes; ++i) words[i][g] = w[i];
      }
      uint8_t* dst = planes + ((i64)(row / kTcM) * nst + st) * kTcABytes + plane_off(row % kTcM, h);
#pragma unroll
      for (int i = 0; i < kPlanes; ++i) {
        uint4 v = make_uint4(words[i][0], words[i][1], words[i][2], words[i][3]);
        *reinterpret_cast<uint4*>(dst + (i64)i * kTcM * kStage) = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// tcgen05, TMEM, bulk copies and mbarriers (inline PTX).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: canonical K-major layout without
// swizzling; leading (K-direction) core-matrix offset 128 bytes, stride
// between 8-row groups 256 bytes; version 1 (bit 46).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait bounded in time; false when the bound (ns) expired first.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// D (TMEM) = A x B^T (acc = 0) or D += A x B^T (acc = 1), N = 32 * nb
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t ad, uint64_t bd, int nb, uint32_t acc) {
  const uint32_t idesc = kTcIdescM | ((uint32_t)(kTcN * nb >> 3) << 17);
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// The MMA schedule of one stage: (plane i of X, first plane j0 of Y, count n).
// The first two write regions 2..9 and 10..15 (levels 13..26, every region
// the epilogue reads) without overlap, so in the first stage of a tile they
// run with acc = 0 and initialise the accumulators; regions 0 and 1 (levels
// 11 and 12) only ever collect what is never read.
struct TcMma {
  int i, j0, n;
};
#define CQR_TC_SCHEDULE                                                                         \
  {13, 0, 8}, {13, 8, 6},                                              /* i = 13: regions 2..9, 10..15 */ \
      {11, 0, 8}, {12, 0, 8},                                          /* i = 11, 12 with all of j = 0..7 */ \
      {3, 8, 6}, {4, 8, 6}, {5, 8, 6}, {6, 8, 6}, {7, 8, 6}, {8, 8, 6}, /* j = 8..13 for 3 <= i <= 12 */ \
      {9, 8, 6}, {10, 8, 6}, {11, 8, 6}, {12, 8, 6},                                                    \
      {6, 7, 1}, {7, 6, 2}, {8, 5, 3}, {9, 4, 4}, {10, 3, 5}, /* j <= 7 with i + j >= 13, i <= 10 */     \
      {2, 11, 3}, {1, 12, 2}, {0, 13, 1}                      /* j >= 11 with i + j >= 13, i <= 2 */
__device__ constexpr TcMma kTcSchedule[22] = {CQR_TC_SCHEDULE};

// Compile-time check of the same entries: every digit pair (i, j) of a kept
// level (i + j >= 13) exactly once, no pair twice, every instruction within
// the planes, N = 32 n <= 256, every region in TMEM, and the first two
// instructions writing each read region (levels 13..26) exactly once and
// nothing else (they run with the accumulate flag off).
constexpr TcMma kTcScheduleCheck[22] = {CQR_TC_SCHEDULE};
constexpr bool tc_schedule_ok() {
  int count[kPlanes][kPlanes] = {};
  int first[kTcCols / kTcN] = {};
  for (int u = 0; u < 22; ++u) {
    const TcMma e = kTcScheduleCheck[u];
    if (e.i < 0 || e.i >= kPlanes || e.j0 < 0 || e.n < 1 || e.j0 + e.n > kPlanes || kTcN * e.n > 256) return false;
    for (int v = 0; v < e.n; ++v) {
      const int j = e.j0 + v, region = e.i + j - kRegionLo;
      if (region < 0 || region >= (int)(kTcCols / kTcN)) return false;
      ++count[e.i][j];
      if (u < 2) ++first[region];
    }
  }
  for (int i = 0; i < kPlanes; ++i)
    for (int j = 0; j < kPlanes; ++j)
      if (count[i][j] > 1 || (i + j >= kLevelLo && count[i][j] != 1)) return false;
  for (int r = 0; r < (int)(kTcCols / kTcN); ++r)
    if (first[r] != (r >= kLevelLo - kRegionLo ? 1 : 0)) return false;
  return true;
}
static_assert(tc_schedule_ok(), "MMA schedule: kept pairs once, regions in range, first two initialise the read regions");
#undef CQR_TC_SCHEDULE
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 8 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tc_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// g * 2^e for an integer |g| < 2^53 (exact), built with integer operations;
// outside the normal range it falls back to the FP64 library ldexp.
__device__ __forceinline__ double scaled_int(long long g, int e) {
  if (g == 0) return 0.0;
  const unsigned long long sgn = g < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long a = g < 0 ? (unsigned long long)(-g) : (unsigned long long)g;
  const int msb = 63 - __clzll((long long)a);
  const int E = msb + e + 1023;
  if (E <= 0 || E >= 2047) return ldexp((double)g, e);
  const unsigned long long mant = (a << (52 - msb)) & 0xFFFFFFFFFFFFFull;
  return __longlong_as_double((long long)(sgn | ((unsigned long long)E << 52) | mant));
}

struct OzArgs {
  const uint8_t* px;  // planes of X (the tile's rows: projection columns p / update rows)
  const uint8_t* py;  // planes of Y (the tile's columns q)
  const int* ex;
  const int* ey;
  int p, q;           // extents (projection: p x q; update: rows of the chunk x N)
  int tiles_p;        // tiles of X in the plane layout (projection: per sub-chunk)
  int y_in_x;         // projection X^T X: the Y tiles are read from the X planes (32-column slices)
  int nst;            // stages per tile (projection: kStagesPerSub)
  int tiles_q;
  int s_off;          // projection: sub-chunk index offset of this launch in the partial buffer
  double* part;       // projection: [s][p * q] column-major p x q
  double* C;          // update: C (ldc) of the chunk's first row
  i64 ldc;
  int* status;
  unsigned long long wait_ns;  // bound of every mbarrier wait (kWaitNs unless the test hook is armed)
  int withhold;                // test hook: the producer issues no copies from this stage on (-1: none)
};

// Projections: one 128 x 32 tile of one sub-chunk per block, grid
// (tiles_q, tiles_p, nsub) with the q tile fastest (the blocks running
// together share the X planes of a sub-chunk in L2); the tile goes to the
// sub-chunk's partial.
__global__ void __launch_bounds__(kTcThreads, 1) ozaki_tc_kernel(OzArgs a) {
  extern __shared__ uint8_t tc_raw[];
  __shared__ __align__(8) uint64_t full_bar[kTcRing], empty_bar[kTcRing], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int give_up;
  if (a.status && *a.status) return;  // uniform across the block, before any allocation
  const int q0 = blockIdx.x * kTcN, p0 = blockIdx.y * kTcM, s = blockIdx.z;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~(uintptr_t)1023);
  // scales of the epilogue, fetched first so that their latency hides behind the contraction
  __shared__ int ey_s[kTcN];
  const int r = 32 * warp + lane;  // tile row = TMEM lane
  const int pr = p0 + r;
  const bool live = pr < a.p;
  const int exr = live ? a.ex[(i64)s * a.p + pr] : kExpZero;
  if (t < kTcN) ey_s[t] = q0 + t < a.q ? a.ey[(i64)s * a.q + q0 + t] : kExpZero;
  if (t == 0) {
    for (int i = 0; i < kTcRing; ++i) {
      mbar_init(smem_u32(&full_bar[i]), 1);
      mbar_init(smem_u32(&empty_bar[i]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    give_up = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int nst = a.nst;
  // this tile's stages: tile-major plane layout, kStagesPerSub stages per (sub-chunk, tile)
  const uint8_t* gx = a.px + ((i64)s * a.tiles_p + p0 / kTcM) * kStagesPerSub * kTcABytes;
  // Y tile: its own planes, or (X^T X) the 32-column slice q0 of the X tile holding it
  const uint8_t* gy = a.y_in_x ? a.px + ((i64)s * a.tiles_p + q0 / kTcM) * kStagesPerSub * kTcABytes +
                                     (i64)(q0 % kTcM) * kStage
                               : a.py + ((i64)s * a.tiles_q + q0 / kTcN) * kStagesPerSub * kTcBBytes;

  if (warp == 0 && lane == 0) {
    // producer: bulk copies of stage st into ring slot st % kTcRing
    int issued = 0;
    for (int st = 0; st < nst; ++st) {
      const int slot = st % kTcRing;
      if (st >= kTcRing && !mbar_wait(smem_u32(&empty_bar[slot]), (uint32_t)((st / kTcRing - 1) & 1), a.wait_ns)) {
        atomicExch(&give_up, 1);
        break;
      }
      if (*(volatile int*)&give_up || st == a.withhold) break;
      const uint32_t fb = smem_u32(&full_bar[slot]);
      const uint32_t sa = smem_u32(ring + slot * kTcStageBytes), sb = sa + kTcABytes;
      mbar_expect_tx(fb, kTcStageBytes);
      bulk_g2s(sa, gx + (i64)st * kTcABytes, kTcABytes, fb);
      if (a.y_in_x) {
#pragma unroll 1
        for (int i = 0; i < kPlanes; ++i)
          bulk_g2s(sb + i * (kTcN * kStage), gy + (i64)st * kTcABytes + i * (kTcM * kStage), kTcN * kStage, fb);
      } else {
        bulk_g2s(sb, gy + (i64)st * kTcBBytes, kTcBBytes, fb);
      }
      issued = st + 1;
    }
    // before leaving, every issued copy must have landed (bounded)
    for (int st = issued - kTcRing < 0 ? 0 : issued - kTcRing; st < issued; ++st)
      mbar_wait(smem_u32(&full_bar[st % kTcRing]), (uint32_t)((st / kTcRing) & 1), a.wait_ns);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: the 22 instructions of each stage (the 105 pairs, level L = i + j into region L - 11)
    for (int st = 0; st < nst; ++st) {
      const int slot = st % kTcRing;
      if (!mbar_wait(smem_u32(&full_bar[slot]), (uint32_t)((st / kTcRing) & 1), a.wait_ns)) {
        atomicExch(&give_up, 1);
        break;
      }
      if (*(volatile int*)&give_up) break;
      tc_fence_after();
      const uint32_t sa = smem_u32(ring + slot * kTcStageBytes), sb = sa + kTcABytes;
      const uint64_t ad0 = tc_desc(sa), bd0 = tc_desc(sb);
#pragma unroll
      for (int u = 0; u < 22; ++u) {
        const TcMma e = kTcSchedule[u];
        const uint64_t ad = ad0 + (uint64_t)((e.i * kTcM * kStage) >> 4);
        const uint64_t bd = bd0 + (uint64_t)((e.j0 * kTcN * kStage) >> 4);
        tc_mma(tmem + (uint32_t)((e.i + e.j0 - kRegionLo) * kTcN), ad, bd, e.n, (st > 0 || u >= 2) ? 1u : 0u);
      }
      tc_commit(smem_u32(&empty_bar[slot]));
    }
    tc_commit(smem_u32(&done_bar));  // arrives when every MMA issued above has completed
  }
  __syncwarp();
  const bool done = mbar_wait(smem_u32(&done_bar), 0, a.wait_ns);
  // one decision for the whole block, and converged warps for tcgen05.ld
  const int failed = __syncthreads_or(!done || *(volatile int*)&give_up);
  tc_fence_after();
  if (failed) {
    if (t == 0 && a.status) atomicCAS(a.status, 0, CQR_STATUS_TIMEOUT);
  } else {
    // epilogue: row r of the tile (TMEM lane r), 8 columns at a time
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
    for (int c0 = 0; c0 < kTcN; c0 += 8) {
      long long g[2][8];
#pragma unroll
      for (int grp = 1; grp >= 0; --grp) {
        uint32_t v[7][8];
#pragma unroll
        for (int l = 6; l >= 0; --l)
          tc_ld8(lane_base + (uint32_t)((kLevelLo - kRegionLo + 7 * grp + l) * kTcN + c0), v[l]);
        tc_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          long long acc = 0;
#pragma unroll
          for (int l = 6; l >= 0; --l) acc = acc * 16 + __float2int_rz(__uint_as_float(v[l][j]));
          g[grp][j] = acc;
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int qc = q0 + c0 + j;
        if (!live || qc >= a.q) continue;
        const int eyc = ey_s[c0 + j];
        double v;
        if (exr == kExpBad || eyc == kExpBad) {
          v = __longlong_as_double(0x7ff8000000000000LL);
        } else if (exr == kExpZero || eyc == kExpZero) {
          v = 0.0;
        } else {
          // sum_L S_L 16^L = 16^13 (g0 + 2^28 g1); value = that * 2^(ex + ey - 112)
          const int e2 = exr + eyc - 112 + 4 * kLevelLo;
          v = scaled_int(g[1][j], e2 + 28) + scaled_int(g[0][j], e2);  // one rounding
        }
        a.part[(i64)(a.s_off + s) * a.p * a.q + pr + (i64)qc * a.p] = v;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

// ---------------------------------------------------------------------------
// Updates C -= X Y as a persistent, warp-specialised kernel: block c takes
// tiles c, c + G, c + 2G, ... (G = grid size; tile T is row tile T / tiles_q,
// column tile T % tiles_q, so the blocks running together share row tiles).
// Warp 0 streams the stages of all its tiles through a three-stage ring, warp
// 1 issues the MMAs of a tile into the one set of TMEM level regions, and
// warps 2-5 (TMEM lane quarters 2, 3, 0, 1) run the epilogue in two phases:
// first the level sums become the exact 64-bit group sums, kept in registers
// (two per column of the thread's row), and the regions are handed back to
// warp 1 at once; then, while the next tile's MMAs run, the group sums are
// scaled, added and subtracted from C.  An update has only K / 32 stages per tile (4 for K = 128), so without
// this overlap the fill and the epilogue would cost as much as the MMAs.
constexpr int kUpRing = 3;
constexpr int kUpThreads = 192;
constexpr int kUpSmem = 1024 + kUpRing * kTcStageBytes;
static_assert(kUpSmem <= kMaxDynSmem, "update ring fits in shared memory");
static_assert(kUpThreads == 6 * 32, "producer, MMA issuer and one epilogue warp per TMEM lane quarter");

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Contraction length up to which every level sum of an update tile is below
// 2^22 in magnitude (14 pairs x 225 x K < 2^22): then the FP32 integer f is
// read exactly as bits(f + 1.5 * 2^23) - bits(1.5 * 2^23), one full-rate
// FP32 add and integer arithmetic, instead of a quarter-rate conversion.
constexpr int kMagicMaxK = 1312;
static_assert(14 * 225 * kMagicMaxK < (1 << 22), "level sums below 2^22");
constexpr float kMagicF = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;  // its encoding

// g = sum_{l<7} s_l 16^l for the seven FP32 level sums v[0..6][j] (s_l
// exact integers, |s_l| < 2^22): three partial sums in unsigned 32-bit
// arithmetic (the offsets cancel modulo 2^32 and |s_0 + 16 s_1 + 256 s_2| <
// 2^31, so the two's-complement reading is the value), then
// g = lo + 2^12 mid + 2^24 s_6.
__device__ __forceinline__ long long group_sum_magic(const uint32_t (&v)[7][8], int j) {
  uint32_t b[7];
#pragma unroll
  for (int l = 0; l < 7; ++l) b[l] = __float_as_uint(__fadd_rn(__uint_as_float(v[l][j]), kMagicF));
  const uint32_t off = 273u * (uint32_t)kMagicBits;  // modulo 2^32
  const int lo = (int)(b[0] + 16u * b[1] + 256u * b[2] - off);
  const int mid = (int)(b[3] + 16u * b[4] + 256u * b[5] - off);
  const int top = (int)(b[6] - (uint32_t)kMagicBits);
  return (long long)lo + ((long long)mid << 12) + ((long long)top << 24);
}

template <bool kMagic>
__global__ void __launch_bounds__(kUpThreads, 1) ozaki_tc_update_kernel(OzArgs a, int ntiles) {
  extern __shared__ uint8_t up_raw[];
  __shared__ __align__(8) uint64_t full_bar[kUpRing], empty_bar[kUpRing], acc_full, acc_empty, mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int give_up;
  if (a.status && *a.status) return;  // uniform across the block, before any allocation
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(up_raw) + 1023) & ~(uintptr_t)1023);
  if (t == 0) {
    for (int i = 0; i < kUpRing; ++i) {
      mbar_init(smem_u32(&full_bar[i]), 1);
      mbar_init(smem_u32(&empty_bar[i]), 1);
    }
    mbar_init(smem_u32(&acc_full), 1);
    mbar_init(smem_u32(&acc_empty), 4);  // one arrival per epilogue warp
    mbar_init(smem_u32(&mma_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    give_up = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int nst = a.nst;

  if (warp == 0) {
    if (lane == 0) {  // producer
      int g = 0;
      bool stop = false;
      for (int T = blockIdx.x; T < ntiles && !stop; T += gridDim.x) {
        // tile-major planes: nst stages per X tile, kStagesPerSub per Y tile
        const uint8_t* gx = a.px + (i64)(T / a.tiles_q) * nst * kTcABytes;
        const uint8_t* gy = a.py + (i64)(T % a.tiles_q) * kStagesPerSub * kTcBBytes;
        for (int st = 0; st < nst; ++st) {
          const int slot = g % kUpRing;
          if (g >= kUpRing && !mbar_wait(smem_u32(&empty_bar[slot]), (uint32_t)((g / kUpRing - 1) & 1), a.wait_ns)) {
            atomicExch(&give_up, 1);
            stop = true;
            break;
          }
          if (*(volatile int*)&give_up || g == a.withhold) {
            stop = true;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[slot]);
          const uint32_t sa = smem_u32(ring + slot * kTcStageBytes), sb = sa + kTcABytes;
          mbar_expect_tx(fb, kTcStageBytes);
          bulk_g2s(sa, gx + (i64)st * kTcABytes, kTcABytes, fb);
          bulk_g2s(sb, gy + (i64)st * kTcBBytes, kTcBBytes, fb);
          ++g;
        }
      }
      // every issued copy must have landed before the block leaves (bounded)
      for (int h = g - kUpRing < 0 ? 0 : g - kUpRing; h < g; ++h)
        mbar_wait(smem_u32(&full_bar[h % kUpRing]), (uint32_t)((h / kUpRing) & 1), a.wait_ns);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      int g = 0, k = 0;
      bool stop = false;
      for (int T = blockIdx.x; T < ntiles && !stop; T += gridDim.x, ++k) {
        if (k >= 1 && !mbar_wait(smem_u32(&acc_empty), (uint32_t)((k - 1) & 1), a.wait_ns)) {
          atomicExch(&give_up, 1);
          break;
        }
        tc_fence_after();
        for (int st = 0; st < nst; ++st) {
          const int slot = g % kUpRing;
          if (!mbar_wait(smem_u32(&full_bar[slot]), (uint32_t)((g / kUpRing) & 1), a.wait_ns) ||
              *(volatile int*)&give_up) {
            atomicExch(&give_up, 1);
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(ring + slot * kTcStageBytes), sb = sa + kTcABytes;
          const uint64_t ad0 = tc_desc(sa), bd0 = tc_desc(sb);
#pragma unroll
          for (int u = 0; u < 22; ++u) {
            const TcMma e = kTcSchedule[u];
            const uint64_t ad = ad0 + (uint64_t)((e.i * kTcM * kStage) >> 4);
            const uint64_t bd = bd0 + (uint64_t)((e.j0 * kTcN * kStage) >> 4);
            tc_mma(tmem + (uint32_t)((e.i + e.j0 - kRegionLo) * kTcN), ad, bd, e.n, (st > 0 || u >= 2) ? 1u : 0u);
          }
          tc_commit(smem_u32(&empty_bar[slot]));
          ++g;
        }
        tc_commit(smem_u32(&acc_full));
      }
      tc_commit(smem_u32(&mma_done));  // every MMA issued above has completed when this arrives
      mbar_wait(smem_u32(&mma_done), 0, a.wait_ns);
    }
  } else {
    // epilogue: TMEM lane quarter qw, tile row r
    const int qw = warp & 3, r = 32 * qw + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * qw) << 16);
    int k = 0;
    for (int T = blockIdx.x; T < ntiles; T += gridDim.x, ++k) {
      const int p0 = (T / a.tiles_q) * kTcM, q0 = (T % a.tiles_q) * kTcN;
      const bool ok = mbar_wait(smem_u32(&acc_full), (uint32_t)(k & 1), a.wait_ns);
      if (!__all_sync(0xffffffffu, ok) || *(volatile int*)&give_up) {
        atomicExch(&give_up, 1);
        break;
      }
      tc_fence_after();
      // phase 1: level sums -> exact group sums g0 (levels 13..19), g1 (20..26), kept in registers
      long long g0[kTcN], g1[kTcN];
#pragma unroll
      for (int c0 = 0; c0 < kTcN; c0 += 8) {
#pragma unroll
        for (int grp = 1; grp >= 0; --grp) {
          uint32_t v[7][8];
#pragma unroll
          for (int l = 6; l >= 0; --l)
            tc_ld8(lane_base + (uint32_t)((kLevelLo - kRegionLo + 7 * grp + l) * kTcN + c0), v[l]);
          tc_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            long long acc = 0;
            if (kMagic) {
              acc = group_sum_magic(v, j);
            } else {
#pragma unroll
              for (int l = 6; l >= 0; --l) acc = acc * 16 + __float2int_rz(__uint_as_float(v[l][j]));
            }
            if (grp) g1[c0 + j] = acc;
            else g0[c0 + j] = acc;
          }
        }
      }
      // hand the regions back to the MMA warp (the next tile's first stage overwrites them)
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acc_empty));
      // phase 2 (overlaps the next tile's MMAs): scale, add the two groups, subtract from C,
      // 16 columns at a time
      const int pr = p0 + r;
      if (pr < a.p) {
        const int exr = a.ex[pr];
#pragma unroll
        for (int h = 0; h < kTcN; h += 16) {
          double cv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) cv[j] = q0 + h + j < a.q ? a.C[pr + (i64)(q0 + h + j) * a.ldc] : 0.0;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int qc = q0 + h + j;
            if (qc >= a.q) continue;
            const int eyc = a.ey[qc];
            double v;
            if (exr == kExpBad || eyc == kExpBad) {
              v = __longlong_as_double(0x7ff8000000000000LL);
            } else if (exr == kExpZero || eyc == kExpZero) {
              v = 0.0;
            } else {
              const int e2 = exr + eyc - 112 + 4 * kLevelLo;
              v = scaled_int(g1[h + j], e2 + 28) + scaled_int(g0[h + j], e2);  // one rounding
            }
            a.C[pr + (i64)qc * a.ldc] = cv[j] - v;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (t == 0 && give_up && a.status) atomicCAS(a.status, 0, CQR_STATUS_TIMEOUT);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
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

void up_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(ozaki_tc_update_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUpSmem);
    cudaFuncSetAttribute(ozaki_tc_update_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUpSmem);
    done = true;
  }
}

void tc_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(ozaki_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    done = true;
  }
}

// One-shot test hook of the bounded waits (cqr_test_arm_wait_expiry): the
// next launch of kernel `g_fault_kernel` (0 = ozaki_tc_kernel, 1 =
// ozaki_tc_update_kernel) gets the armed stage to withhold and wait bound,
// then the hook disarms itself.
std::mutex g_fault_mu;
int g_fault_kernel = -1, g_fault_stage = -1;
unsigned long long g_fault_ns = 0;

void take_fault(int kernel, OzArgs& a) {
  a.wait_ns = kWaitNs;
  a.withhold = -1;
  std::lock_guard<std::mutex> lk(g_fault_mu);
  if (g_fault_kernel == kernel) {
    a.wait_ns = g_fault_ns;
    a.withhold = g_fault_stage;
    g_fault_kernel = -1;
  }
}

// Rows per update chunk: the X planes of one chunk take about 1 GiB.
inline i64 oz_nn_rows(int nst) {
  i64 rows = ((i64)1 << 30) / ((i64)kPlanes * kStage * nst);
  rows = rows / kTcM * kTcM;
  return rows < kTcM ? kTcM : rows;
}

}  // namespace

// Rows per splitting chunk of a projection: planes of one chunk take 1 to
// 2 GiB.  A launch has (column tiles) x (sub-chunks) blocks of equal length,
// one per SM, so a partly filled last wave costs a whole one; of the
// sub-chunk counts between the 1 GiB budget and twice it, the one with the
// fewest waves per sub-chunk is taken (the smallest among equals).
i64 oz_chunk_rows(int p, int q) {
  const i64 cpx = round_up(p, kTcM), cpy = round_up(q, kTcN);
  i64 base = ((i64)1 << 30) / ((i64)kPlanes * (cpx + cpy) * kSub);
  if (base < 1) base = 1;
  const i64 tiles = (cpx / kTcM) * (cpy / kTcN);
  i64 best = base;
  for (i64 n = base + 1; n <= 2 * base; ++n) {
    // waves(n) / n < waves(best) / best, in integers
    const i64 wn = (tiles * n + kSMs - 1) / kSMs, wb = (tiles * best + kSMs - 1) / kSMs;
    if (wn * best < wb * n) best = n;
  }
  return best * kSub;
}

size_t ozaki_workspace_bytes(i64 m, int p, int q) {
  if (m <= 0 || p <= 0 || q <= 0) return 0;
  const int cpx = round_up(p, kTcM), cpy = round_up(q, kTcN);
  const i64 nsub_total = (m + kSub - 1) / kSub;
  i64 ch = oz_chunk_rows(p, q);
  const i64 mr = nsub_total * kSub;
  if (ch > mr) ch = mr;
  const i64 nsub_ch = ch / kSub;
  size_t b = 0;
  b += (size_t)nsub_ch * kPlanes * (cpx + cpy) * kSub;        // planes of one chunk
  b = (b + 255) & ~(size_t)255;
  b += sizeof(int) * (size_t)nsub_ch * (p + q);               // scales
  b = (b + 255) & ~(size_t)255;
  b += sizeof(double) * (size_t)nsub_total * p * q;           // partials
  return (b + 255) & ~(size_t)255;
}

cudaError_t tn_product_emulated(i64 m, int p, int q, const double* X, i64 ldx, const double* Y, i64 ldy,
                                void* ws, double* C, i64 ldc, const int* status, cudaStream_t st) {
  if (p <= 0 || q <= 0) return cudaSuccess;
  const int cpx = round_up(p, kTcM), cpy = round_up(q, kTcN);
  const i64 nsub_total = (m + kSub - 1) / kSub;
  i64 ch = oz_chunk_rows(p, q);
  const i64 mr = nsub_total * kSub;
  if (ch > mr) ch = mr;
  const i64 nsub_ch = ch / kSub;
  uint8_t* planes = (uint8_t*)ws;
  size_t off = (size_t)nsub_ch * kPlanes * (cpx + cpy) * kSub;
  off = (off + 255) & ~(size_t)255;
  int* exps = (int*)((char*)ws + off);
  off += sizeof(int) * (size_t)nsub_ch * (p + q);
  off = (off + 255) & ~(size_t)255;
  double* part = (double*)((char*)ws + off);
  tc_attr();
  uint8_t* px = planes;
  uint8_t* py = planes + (size_t)nsub_ch * kPlanes * cpx * kSub;
  int* ex = exps;
  int* ey = exps + nsub_ch * p;
  const int tiles_p = cpx / kTcM, tiles_q = cpy / kTcN;
  const bool same = X == Y && ldx == ldy && p == q;  // X^T X: split once
  for (i64 r0 = 0; r0 < m; r0 += ch) {
    const i64 nsub = ((m - r0 < ch ? m - r0 : ch) + kSub - 1) / kSub;
    prof_begin(kMisc, st);
    ozaki_split_kernel<<<dim3((unsigned)((p + 7) / 8), (unsigned)nsub), 256, 0, st>>>(X, ldx, m, r0, p, kTcM, px, ex, status);
    prof_end(kMisc, 0.0, st);
    if (!same) {
      prof_begin(kMisc, st);
      ozaki_split_kernel<<<dim3((unsigned)((q + 7) / 8), (unsigned)nsub), 256, 0, st>>>(Y, ldy, m, r0, q, kTcN, py, ey, status);
      prof_end(kMisc, 0.0, st);
    }
    OzArgs a{};
    a.px = px;
    a.py = same ? px : py;
    a.ex = ex;
    a.ey = same ? ex : ey;
    a.p = p;
    a.q = q;
    a.tiles_p = tiles_p;
    a.y_in_x = same ? 1 : 0;
    a.nst = kStagesPerSub;
    a.tiles_q = tiles_q;
    a.s_off = (int)(r0 / kSub);
    a.part = part;
    a.status = const_cast<int*>(status);
    take_fault(0, a);
    prof_begin(kProjection, st);
    ozaki_tc_kernel<<<dim3((unsigned)tiles_q, (unsigned)tiles_p, (unsigned)nsub), kTcThreads, kTcSmem, st>>>(a);
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
  const int cpy = round_up(N, kTcN);
  i64 rows = oz_nn_rows(nst);
  const i64 mr = (M + kTcM - 1) / kTcM * kTcM;
  if (rows > mr) rows = mr;
  size_t b = (size_t)rows * nst * kStage * kPlanes;  // X planes of one chunk
  b = (b + 255) & ~(size_t)255;
  b += (size_t)kSub * kPlanes * cpy;                 // Y planes (one sub-chunk)
  b = (b + 255) & ~(size_t)255;
  b += sizeof(int) * ((size_t)rows + N);             // scales
  return (b + 255) & ~(size_t)255;
}

cudaError_t nn_update_emulated(i64 M, int N, int K, const double* X, i64 ldx, const double* Y, i64 ldy, double* C,
                               i64 ldc, void* ws, const int* status, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  const int kcmax = K < kSub ? K : kSub;
  const int nstmax = (kcmax + kStage - 1) / kStage;
  const int cpy = round_up(N, kTcN);
  i64 rows = oz_nn_rows(nstmax);
  const i64 mr = (M + kTcM - 1) / kTcM * kTcM;
  if (rows > mr) rows = mr;
  uint8_t* px = (uint8_t*)ws;
  size_t off = ((size_t)rows * nstmax * kStage * kPlanes + 255) & ~(size_t)255;
  uint8_t* py = (uint8_t*)ws + off;
  off = (off + (size_t)kSub * kPlanes * cpy + 255) & ~(size_t)255;
  int* ex = (int*)((char*)ws + off);
  int* ey = ex + rows;
  up_attr();
  const int tiles_q = cpy / kTcN;
  for (i64 k0 = 0; k0 < K; k0 += kSub) {
    const int kc = (int)(K - k0 < kSub ? K - k0 : kSub);
    const int nst = (kc + kStage - 1) / kStage;
    prof_begin(kMisc, st);
    ozaki_split_kernel<<<dim3((unsigned)((N + 7) / 8), 1u), 256, 0, st>>>(Y, ldy, k0 + kc, k0, N, kTcN, py, ey, status);
    prof_end(kMisc, 0.0, st);
    for (i64 r0 = 0; r0 < M; r0 += rows) {
      const i64 live = M - r0 < rows ? M - r0 : rows;
      const int rws = (int)((live + kTcM - 1) / kTcM * kTcM);
      prof_begin(kMisc, st);
      ozaki_rowsplit_kernel<<<(unsigned)(rws / 128), 128, 0, st>>>(X, ldx, M, r0, rws, k0, kc, px, ex, status);
      prof_end(kMisc, 0.0, st);
      OzArgs a{};
      a.px = px;
      a.py = py;
      a.ex = ex;
      a.ey = ey;
      a.p = (int)live;
      a.q = N;
      a.tiles_p = rws / kTcM;
      a.nst = nst;
      a.tiles_q = tiles_q;
      a.C = C + r0;
      a.ldc = ldc;
      a.status = const_cast<int*>(status);
      take_fault(1, a);
      const int ntiles = (rws / kTcM) * tiles_q;
      prof_begin(kUpdate, st);
      const unsigned grid = (unsigned)(ntiles < kSMs ? ntiles : kSMs);
      if (nst * kStage <= kMagicMaxK)
        ozaki_tc_update_kernel<true><<<grid, kUpThreads, kUpSmem, st>>>(a, ntiles);
      else
        ozaki_tc_update_kernel<false><<<grid, kUpThreads, kUpSmem, st>>>(a, ntiles);
      prof_end(kUpdate, 2.0 * (double)live * N * kc, st);
    }
  }
  return cudaGetLastError();
}

}  // namespace cqr

extern "C" int cqr_test_arm_wait_expiry(int kernel, int stage, long long wait_ns) {
  if (kernel < -1 || kernel > 1) return -1;
  if (kernel == -1) {  // disarm
    std::lock_guard<std::mutex> lk(cqr::g_fault_mu);
    cqr::g_fault_kernel = -1;
    return 0;
  }
  if (stage < 0) return -2;
  if (wait_ns < 1 || wait_ns > (long long)cqr::kWaitNs) return -3;
  std::lock_guard<std::mutex> lk(cqr::g_fault_mu);
  cqr::g_fault_kernel = kernel;
  cqr::g_fault_stage = stage;
  cqr::g_fault_ns = (unsigned long long)wait_ns;
  return 0;
}
