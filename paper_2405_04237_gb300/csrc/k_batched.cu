// Persistent batched mCQR2GS (Alg. 9) for many small tall-skinny matrices
// (n <= 128) in ONE cooperative launch.
//
// Work split.  The grid holds one CTA of kBT threads per SM, all resident
// (cooperative launch).  CTAs form groups of G consecutive blocks; group g
// factors, one after the other, the matrices of its list (a static
// largest-first schedule computed on the host).  Inside a group the rows of
// the current matrix are split into G contiguous ranges, one per CTA: this
// is the paper's 1-D row-block distribution (Alg. 2, Alg. 8) with the G
// CTAs as the ranks.  Every step that sums over the m rows ends with each
// CTA writing its partial sum to its own slot, a group barrier, and every
// CTA adding the G slots in rank order and doing the small dense work (the
// b x b Cholesky, the triangular products) redundantly -- the "Allreduce +
// redundant Cholesky" of Alg. 2 -- so all CTAs of a group hold bitwise
// identical factors without a second barrier.
//
// Passes.  One panel step of Alg. 9 reads the rows it needs once per pass,
// in sub-blocks of 64 to 256 rows (more when fewer columns are loaded)
// staged in shared memory, and fuses the
// streaming operation with the next m-row sum:
//   first pass    (copy A -> Q if out of place) + Gram of panel 1
//   T1            Q_j = A_j S1^{-1}  + Gram (j = 1) or Z = Q_{1:j-1}^T P (j > 1)
//   RO  (j > 1)   P -= Q_{1:j-1} Z   + Gram of P
//   T2            Q_j = P S2^{-1}    + Y = Q_j^T A_{j+1:k}
//   U   (j > 1)   A_{j:k} -= Q_{j-1} Y + Gram of the new panel A_j
// with the reductions between them.  R is assembled by the ranks, column
// slices each: R_jj = S2 S1, R_{1:j-1,j} += Z S1, R_{j,j+1:k} = Y.
//
// Adaptive panel width (optional, per launch): the first CholeskyQR of each
// panel is tested like CQR_HALVE of the single-matrix path -- a breakdown or
// (max U_ii / min U_ii)^2 > 1/(64 u) rejects the panel, whose Gram matrix is
// then formed again for the largest divisor of b that is <= b/2 -- all on
// the device, every CTA of the group taking the same decision.
//
// Failure handling.  A Cholesky breakdown sets the matrix's status to its
// global column + 1 and the group moves on.  Every group-barrier wait is
// bounded in time (kBWaitNs of the global timer); on expiry the CTA raises
// the launch-wide abort flag, every group marks its current and remaining
// matrices CQR_STATUS_TIMEOUT and returns.  A one-shot host-side hook makes
// one CTA skip one barrier arrival so that this path can be tested.
#include <algorithm>
#include <string.h>

#include <mutex>
#include <vector>

#include "cqr.h"
#include "cqr_common.cuh"

#define TRY_RET(x)                    \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

namespace cqr {

namespace {

constexpr int kBT = 512;            // threads per CTA
constexpr int kBR = 64;             // rows per staged sub-block at full width (multiples of it below)
constexpr int kBRMax = 4 * kBR;     // rows per staged sub-block for narrow passes
constexpr int kBNMax = 128;         // widest matrix of the persistent path
constexpr int kBSlot = 8448;        // doubles per partial slot: the Gram of b = 128 (528 tiles x 16)
constexpr unsigned long long kBWaitNs = 2000000000ull;
static_assert(kBSlot >= 528 * 16 && kBSlot >= (kBNMax / 2) * (kBNMax / 2), "a slot holds any partial");

struct BMat {
  const double* A;
  double* Q;
  double* R;
  i64 m, lda;   // ldq = lda, ldr = n
  int n, b;     // width, starting panel width
};

struct BArgs {
  const BMat* mats;
  const int* order;    // matrices of group g: order[gstart[g] .. gstart[g+1])
  const int* gstart;
  int* status;         // per matrix
  int* bfinal;         // per matrix: width of its last panel
  double* part;        // [2][gridDim.x][kBSlot]
  double* s1;          // [groups][kBNMax * kBNMax]: S1 of the current panel (column-major)
  unsigned int* bar;   // [groups] barrier counters (zero at launch)
  int* abort;          // launch-wide abort flag (zero at launch)
  int G;               // CTAs per group
  int nmax, bmax;      // shared-memory layout
  int halve;           // adaptive panel width
  unsigned long long wait_ns;
  int hook_group, hook_rank, hook_barrier;  // test hook: that CTA skips that barrier's arrival
};

// Shared memory (doubles): tile [kBR][ts] (ts = nmax + 1, odd) or the
// reduction scratch [kBT][16]; U [bmax * bmax] row-major (zero diagonal and
// lower triangle once factored); dg, rv [bmax]; M [nmax^2/4] (Y or Z).
struct Smem {
  double* tile;
  double* red;
  double* U;
  double* dg;
  double* rv;
  double* M;
  int ts;   // row stride of the staged tile (set per pass)
  int rb;   // rows of the staged tile (set per pass, a multiple of kBR)
};

__host__ __device__ inline int tile_stride(int nmax) { return nmax + 1; }
__host__ __device__ inline size_t region0_doubles(int nmax) {
  const size_t t = (size_t)kBR * tile_stride(nmax), r = (size_t)kBT * 16;
  return t > r ? t : r;
}
__host__ __device__ inline size_t mdoubles(int nmax) { return (size_t)nmax * nmax / 4 + 1; }
size_t bsmem_bytes(int nmax, int bmax) {
  return sizeof(double) * (region0_doubles(nmax) + (size_t)bmax * bmax + 2 * (size_t)bmax + mdoubles(nmax));
}

__device__ Smem carve(double* sm, int nmax, int bmax) {
  Smem s;
  s.tile = sm;
  s.red = sm;
  s.U = sm + region0_doubles(nmax);
  s.dg = s.U + (size_t)bmax * bmax;
  s.rv = s.dg + bmax;
  s.M = s.rv + bmax;
  s.ts = tile_stride(nmax);
  s.rb = kBR;
  return s;
}

__device__ __forceinline__ unsigned long long bglobal_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// 8-byte asynchronous global -> shared copy; zero-fills when !valid (the
// source is then not read).
__device__ __forceinline__ void cp_async8(double* dst, const double* src, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sa), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// Group barrier, bounded in time.  Returns false (for every thread of the
// CTA) when the wait expired or another CTA raised the abort flag.
__device__ bool group_barrier(const BArgs& a, int group, int rank, unsigned int* count, int* ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int c = ++(*count);
    int good = 1;
    __threadfence();  // this CTA's partial sums and R columns before the arrival
    const bool skip = group == a.hook_group && rank == a.hook_rank && (int)c == a.hook_barrier;
    if (!skip) atomicAdd(&a.bar[group], 1u);
    const unsigned int target = c * (unsigned int)a.G;
    const unsigned long long t0 = bglobal_ns();
    while (ld_acquire(&a.bar[group]) < target) {
      if (*(volatile int*)a.abort) {
        good = 0;
        break;
      }
      if (bglobal_ns() - t0 > a.wait_ns) {
        atomicExch(a.abort, 1);
        good = 0;
        break;
      }
    }
    __threadfence();
    *ok = good;
  }
  __syncthreads();
  return *ok != 0;
}

// ---------------------------------------------------------------------------
// Transposed products over a staged sub-block: C (p x q) += X^T Y, X and Y
// column ranges of the tile.  The output is cut into 4 x 4 tiles (for the
// Gram matrix only the tiles on or above the diagonal).  The largest power
// of two M <= (tile count) of them are "main" tiles, each owned by kBT / M
// threads that split the rows round-robin; the remaining E are "extra"
// tiles, each owned by kBT / E threads that also split the rows.  Every
// thread thus has one main and at most one extra 4 x 4 accumulator, and the
// threads of a warp run the same instruction stream.
struct TnMap {
  int sym;        // Gram: upper tiles of a T x T grid
  int tp, cnt;    // tiles along p (TN), tile count
  int M, RG;      // main tiles, row groups
  int E, tpt;     // extra tiles, threads per extra tile
  int xc, yc;     // tile columns of X and Y
};

__device__ __forceinline__ void tile_ij(const TnMap& mp, int id, int& i, int& j) {
  if (mp.sym) {
    int jj = (int)((sqrtf(8.0f * (float)id + 1.0f) - 1.0f) * 0.5f);
    while ((jj + 1) * (jj + 2) / 2 <= id) ++jj;
    while (jj * (jj + 1) / 2 > id) --jj;
    j = jj;
    i = id - jj * (jj + 1) / 2;
  } else {
    i = id % mp.tp;
    j = id / mp.tp;
  }
}

__device__ TnMap make_map(int sym, int p, int q, int xc, int yc) {
  TnMap mp;
  mp.sym = sym;
  mp.tp = p / 4;
  const int tq = q / 4;
  mp.cnt = sym ? mp.tp * (mp.tp + 1) / 2 : mp.tp * tq;
  int M = 1;
  while (M * 2 <= mp.cnt && M * 2 <= kBT) M *= 2;
  mp.M = M;
  mp.RG = kBT / M;
  mp.E = mp.cnt - M;
  mp.tpt = mp.E > 0 ? kBT / mp.E : 0;
  mp.xc = xc;
  mp.yc = yc;
  return mp;
}

__device__ __forceinline__ void acc_tile(const double* tile, int ts, int r, int xc, int yc, double (&acc)[4][4]) {
  const double* row = tile + (size_t)r * ts;
  double x[4], y[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    x[u] = row[xc + u];
    y[u] = row[yc + u];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = fma(x[u], y[v], acc[u][v]);
}

// accumulate one staged sub-block (kBR rows, zero beyond the live rows)
__device__ __forceinline__ void tn_accumulate(const TnMap& mp, const Smem& s, int nr, double (&am)[4][4],
                                              double (&ae)[4][4]) {
  const int t = threadIdx.x;
  {
    int i, j;
    tile_ij(mp, t % mp.M, i, j);
    const int xc = mp.xc + 4 * i, yc = mp.yc + 4 * j;
    for (int r = t / mp.M; r < nr; r += mp.RG) acc_tile(s.tile, s.ts, r, xc, yc, am);
  }
  if (mp.E > 0 && t < mp.E * mp.tpt) {
    int i, j;
    tile_ij(mp, mp.M + t / mp.tpt, i, j);
    const int xc = mp.xc + 4 * i, yc = mp.yc + 4 * j;
    for (int r = t % mp.tpt; r < nr; r += mp.tpt) acc_tile(s.tile, s.ts, r, xc, yc, ae);
  }
}

// In-CTA sums of the accumulators in a fixed order (row groups, then the
// threads of an extra tile in thread order), written tile-major (16 doubles
// per tile, entry u * 4 + v) to this CTA's slot.
__device__ void tn_flush(const TnMap& mp, const Smem& s, double (&am)[4][4], double (&ae)[4][4], double* slot) {
  const int t = threadIdx.x;
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) s.red[(size_t)t * 16 + u * 4 + v] = am[u][v];
  __syncthreads();
  if (t < mp.M) {
    for (int e = 0; e < 16; ++e) {
      double sum = 0.0;
      for (int g = 0; g < mp.RG; ++g) sum += s.red[(size_t)(g * mp.M + t) * 16 + e];
      slot[(size_t)t * 16 + e] = sum;
    }
  }
  __syncthreads();
  if (mp.E > 0) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) s.red[(size_t)t * 16 + u * 4 + v] = ae[u][v];
    __syncthreads();
    if (t < mp.E * mp.tpt && t % mp.tpt == 0) {
      for (int e = 0; e < 16; ++e) {
        double sum = 0.0;
        for (int k = 0; k < mp.tpt; ++k) sum += s.red[(size_t)(t + k) * 16 + e];
        slot[(size_t)(mp.M + t / mp.tpt) * 16 + e] = sum;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// C (tile columns [cc, cc+q)) -= X (tile columns [xc, xc+p)) * Mm (p x q,
// row-major, leading dimension q), in place in the staged sub-block.  Each
// thread owns a TR x TC block of C (the shape that keeps the most threads
// busy, a template so that no multiply-add is issued for padding); the sum
// starts from C and takes one fused multiply-add per term in ascending k.
template <int TR, int TC>
__device__ void nn_update_block(const Smem& s, int nr, int xc, int p, int cc, int q, const double* Mm) {
  const int nrt = s.rb / TR;
  const int nblk = nrt * (q / TC);
  for (int bi = threadIdx.x; bi < nblk; bi += kBT) {
  const int r0 = (bi % nrt) * TR, c0 = (bi / nrt) * TC;
  if (r0 >= nr) continue;  // padding rows only
  double acc[TR][TC];
#pragma unroll
  for (int u = 0; u < TR; ++u)
#pragma unroll
    for (int v = 0; v < TC; ++v) acc[u][v] = s.tile[(size_t)(r0 + u) * s.ts + cc + c0 + v];
#pragma unroll 2
  for (int k = 0; k < p; ++k) {
    double x[TR], mv[TC];
#pragma unroll
    for (int u = 0; u < TR; ++u) x[u] = s.tile[(size_t)(r0 + u) * s.ts + xc + k];
#pragma unroll
    for (int v = 0; v < TC; ++v) mv[v] = Mm[(size_t)k * q + c0 + v];
#pragma unroll
    for (int u = 0; u < TR; ++u)
#pragma unroll
      for (int v = 0; v < TC; ++v) acc[u][v] = fma(-x[u], mv[v], acc[u][v]);
  }
#pragma unroll
  for (int u = 0; u < TR; ++u)
#pragma unroll
    for (int v = 0; v < TC; ++v) s.tile[(size_t)(r0 + u) * s.ts + cc + c0 + v] = acc[u][v];
  }
}

__device__ void nn_update(const Smem& s, int nr, int xc, int p, int cc, int q, const double* Mm) {
  // the candidate shape with the most threads <= kBT (ties: the larger block);
  // 4 x 4 always fits (staged rows x loaded width <= the staging area)
  int best = -1, pick = 7;
  const int cand[8][2] = {{4, 4}, {4, 3}, {4, 2}, {2, 3}, {4, 1}, {1, 3}, {2, 1}, {1, 1}};
  for (int k = 0; k < 8; ++k) {
    if (q % cand[k][1]) continue;
    const int thr = (s.rb / cand[k][0]) * (q / cand[k][1]);
    if (thr <= kBT && thr > best) {
      best = thr;
      pick = k;
    }
  }
  switch (pick) {
    case 0: nn_update_block<4, 4>(s, nr, xc, p, cc, q, Mm); break;
    case 1: nn_update_block<4, 3>(s, nr, xc, p, cc, q, Mm); break;
    case 2: nn_update_block<4, 2>(s, nr, xc, p, cc, q, Mm); break;
    case 3: nn_update_block<2, 3>(s, nr, xc, p, cc, q, Mm); break;
    case 4: nn_update_block<4, 1>(s, nr, xc, p, cc, q, Mm); break;
    case 5: nn_update_block<1, 3>(s, nr, xc, p, cc, q, Mm); break;
    case 6: nn_update_block<2, 1>(s, nr, xc, p, cc, q, Mm); break;
    default: nn_update_block<1, 1>(s, nr, xc, p, cc, q, Mm); break;
  }
}

// Row-wise forward substitution on tile columns [tc, tc+b): with the rows
// of U pre-scaled by the reciprocal diagonal (Ut_cc' = U_cc' / U_cc, see
// prescale_rows), s_c' -= s_c Ut_cc' for c' > c in ascending c, then
// q_c = s_c / U_cc (by the reciprocal rv[c]) -- q_c U_cc' = s_c Ut_cc', so
// this is the substitution q_c = (x_c - sum_{i<c} q_i U_ic) / U_cc with
// the division moved past the products.  L lanes of one warp share a row;
// lane l owns the columns c = l (mod L).  Rows >= nr (padding) are skipped.
__device__ void trsm_rows_staged(const Smem& s, int tc, int b, int nr) {
  int L = kBT / s.rb;  // lanes per row: every thread busy, at most 8, at most b
  L = L > 8 ? 8 : L;
  L = L > b ? b : L;
  const int t = threadIdx.x;
  const int r = t / L, l = t % L;
  const bool active = t < s.rb * L && r < nr;
  double* row = s.tile + (size_t)r * s.ts + tc;
  for (int c = 0; c < b; ++c) {
    __syncwarp();  // column c complete: its last update came at step c - 1
    if (active) {
      const double q = row[c];
      const double* urow = s.U + (size_t)c * b;
      for (int cp = (c + 1) / L * L + l; cp < b; cp += L)
        if (cp > c) row[cp] = fma(-q, urow[cp], row[cp]);
    }
  }
  __syncwarp();
  if (active)
    for (int c = l; c < b; c += L) row[c] *= s.rv[c];
}

// U_cc' := U_cc' / U_cc (by the reciprocal) for c' > c: the form the staged
// substitution uses.  Called after the unscaled factor has been used for
// the R products and saved.
__device__ void prescale_rows(const Smem& s, int b) {
  for (int e = threadIdx.x; e < b * b; e += kBT) {
    const int c = e / b, cp = e % b;
    if (cp > c) s.U[e] *= s.rv[c];
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// One pass over this CTA's rows [R0, R1) of a matrix.
struct PassSpec {
  const double* src;  // rows come from here (A or Q), leading dimension lds
  i64 lds;
  double* dst;        // written-back columns go here (Q), leading dimension ldd
  i64 ldd;
  int lo, hi;         // loaded columns (tile column = column - lo)
  int st_lo, st_hi;   // written-back columns
  int op1;            // 0 none, 1 trsm on [t0, t0+tb), 2 update C[c0u, c0u+qu) -= X[x0u, x0u+pu) Mm
  int t0, tb;
  int x0u, pu, c0u, qu;
  const double* Mm;
  int op2;            // 0 none, 1 Gram of [g0, g0+gb), 2 X^T Y with X [x0, x0+px), Y [y0, y0+qy)
  int g0, gb;
  int x0, px, y0, qy;
};

__device__ void run_pass(const PassSpec& P, const Smem& s0, i64 R0, i64 R1, double* slot) {
  const int t = threadIdx.x;
  // the tile for this pass: an odd row stride just above the loaded width,
  // and as many 64-row groups (up to 4) as the staging area holds
  Smem s = s0;
  {
    const int w = P.hi - P.lo;
    s.ts = (w % 2 == 0) ? w + 1 : w + 2;
    const int fit = (int)(region0_doubles(s0.ts - 1) / ((size_t)kBR * s.ts));
    int groups = 1;  // 1, 2 or 4 groups of 64 rows, so that the solve's lanes x rows fill the block
    while (groups * 2 <= fit && groups * 2 <= kBRMax / kBR) groups *= 2;
    s.rb = groups * kBR;
  }
  TnMap mp{};
  if (P.op2 == 1) mp = make_map(1, P.gb, P.gb, P.g0 - P.lo, P.g0 - P.lo);
  if (P.op2 == 2) mp = make_map(0, P.px, P.qy, P.x0 - P.lo, P.y0 - P.lo);
  double am[4][4], ae[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) am[u][v] = ae[u][v] = 0.0;
  const int w = P.hi - P.lo;
  const int rb = s.rb;
  for (i64 r0 = R0; r0 < R1; r0 += rb) {
    const int nr = (int)imin64(rb, R1 - r0);
    // stage rows (zero beyond nr): asynchronous copies, coalesced along the
    // rows of each column, all in flight before the one wait
    for (int e = t; e < rb * w; e += kBT) {
      const int r = e % rb, c = e / rb;
      const bool ok = r < nr;
      cp_async8(s.tile + (size_t)r * s.ts + c, ok ? P.src + (r0 + r) + (i64)(P.lo + c) * P.lds : P.src, ok);
    }
    cp_async_wait_all();
    __syncthreads();
    if (P.op1 == 1) trsm_rows_staged(s, P.t0 - P.lo, P.tb, nr);
    if (P.op1 == 2) nn_update(s, nr, P.x0u - P.lo, P.pu, P.c0u - P.lo, P.qu, P.Mm);
    __syncthreads();
    const int ws = P.st_hi - P.st_lo;
    for (int e = t; e < rb * ws; e += kBT) {
      const int r = e % rb, c = e / rb;
      if (r < nr) P.dst[(r0 + r) + (i64)(P.st_lo + c) * P.ldd] = s.tile[(size_t)r * s.ts + (P.st_lo - P.lo) + c];
    }
    if (P.op2) tn_accumulate(mp, s, nr, am, ae);
    __syncthreads();
  }
  if (P.op2) tn_flush(mp, s, am, ae, slot);
}

// Sum of the G slots of the group (rank order) for output entry (a, c).
__device__ __forceinline__ double slot_sum(const double* slots, int G, int sym, int tp, int a, int c) {
  const int i = a / 4, j = c / 4;
  const int id = sym ? j * (j + 1) / 2 + i : i + j * tp;
  const double* p = slots + (size_t)id * 16 + (a % 4) * 4 + (c % 4);
  double v = 0.0;
  int g = 0;
  for (; g + 4 <= G; g += 4) {  // four loads in flight, added in rank order
    const double x0 = p[(size_t)g * kBSlot], x1 = p[(size_t)(g + 1) * kBSlot];
    const double x2 = p[(size_t)(g + 2) * kBSlot], x3 = p[(size_t)(g + 3) * kBSlot];
    v += x0;
    v += x1;
    v += x2;
    v += x3;
  }
  for (; g < G; ++g) v += p[(size_t)g * kBSlot];
  return v;
}

// W = sum of the slots (upper triangle), then the right-looking Cholesky
// W = U^T U in shared memory.  Returns the local breakdown column or -1;
// *rej (when the panel test is on and b > 1) = breakdown or
// (max U_jj / min U_jj)^2 > 1/(64 u).  Leaves U with zero diagonal and
// lower triangle in s.U, the diagonal in s.dg and its reciprocals in s.rv.
__device__ int reduce_cholesky(const Smem& s, const double* slots, int G, int b, bool test, int* rej,
                               int* sh_broken) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = kBT / 32;
  double* U = s.U;
  for (int e = t; e < b * b; e += kBT) {
    const int a = e / b, c = e % b;
    U[e] = a <= c ? slot_sum(slots, G, 1, 0, a, c) : 0.0;
  }
  if (t == 0) *sh_broken = -1;
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (warp == 0) {
      const double d = U[(size_t)j * b + j];
      if (d > 0.0 && isfinite(d)) {
        const double u = sqrt(d);
        for (int c = j + 1 + lane; c < b; c += 32) U[(size_t)j * b + c] /= u;
        if (lane == 0) {
          U[(size_t)j * b + j] = u;
          s.dg[j] = u;
          s.rv[j] = 1.0 / u;
        }
      } else if (lane == 0) {
        *sh_broken = j;
      }
    }
    __syncthreads();
    if (*sh_broken >= 0) break;
    for (int a = j + 1 + warp; a < b; a += nw) {
      const double ua = U[(size_t)j * b + a];
      for (int c = a + lane; c < b; c += 32) U[(size_t)a * b + c] = fma(-ua, U[(size_t)j * b + c], U[(size_t)a * b + c]);
    }
    __syncthreads();
  }
  const int broken = *sh_broken;
  if (test && t == 0) {
    int r = 0;
    if (b > 1) {
      if (broken >= 0) {
        r = 1;
      } else {
        double dmax = s.dg[0], dmin = s.dg[0];
        for (int j = 1; j < b; ++j) {
          dmax = s.dg[j] > dmax ? s.dg[j] : dmax;
          dmin = s.dg[j] < dmin ? s.dg[j] : dmin;
        }
        r = dmax * dmax * 64.0 * 0x1p-53 > dmin * dmin;
      }
    }
    *rej = r;
  }
  __syncthreads();
  if (broken < 0)  // the solve's form: zero diagonal (its reciprocal is in rv)
    for (int e = t; e < b; e += kBT) U[(size_t)e * b + e] = 0.0;
  __syncthreads();
  return broken;
}

// M = sum of the slots: a p x q transposed product, row-major in s.M.
__device__ void reduce_tn(const Smem& s, const double* slots, int G, int p, int q) {
  for (int e = threadIdx.x; e < p * q; e += kBT) {
    const int a = e / q, c = e % q;
    s.M[e] = slot_sum(slots, G, 0, p / 4, a, c);
  }
  __syncthreads();
}

// S (b x b upper, with diagonal) element (a, c) from the staged factor.
__device__ __forceinline__ double su(const Smem& s, int b, int a, int c) {
  return a == c ? s.dg[a] : s.U[(size_t)a * b + c];
}

__device__ int halved(int b) {
  for (int d = b / 2; d > 1; --d)
    if (b % d == 0) return d;
  return 1;
}

__global__ void __launch_bounds__(kBT, 1) batched_mcqr2gs_kernel(BArgs a) {
  extern __shared__ __align__(16) double bsm[];
  __shared__ unsigned int bar_count;
  __shared__ int bar_ok, sh_broken, sh_rej;
  const Smem s = carve(bsm, a.nmax, a.bmax);
  const int t = threadIdx.x;
  const int group = blockIdx.x / a.G, rank = blockIdx.x % a.G;
  if (t == 0) bar_count = 0;
  __syncthreads();
  double* slots[2] = {a.part + (size_t)(0 * gridDim.x + group * a.G) * kBSlot,
                      a.part + (size_t)(1 * gridDim.x + group * a.G) * kBSlot};
  int phase = 0;  // partial buffer parity
  double* s1g = a.s1 + (size_t)group * kBNMax * kBNMax;
  const int l0 = a.gstart[group], l1 = a.gstart[group + 1];
  bool alive = true;
  int li = l0;
  for (; li < l1 && alive; ++li) {
    if (*(volatile int*)a.abort) {
      alive = false;
      break;
    }
    const int mi = a.order[li];
    const BMat mt = a.mats[mi];
    const int n = mt.n;
    const i64 R0 = (i64)rank * mt.m / a.G, R1 = (i64)(rank + 1) * mt.m / a.G;
    const bool oop = mt.Q != mt.A;
    // zero R (column slices of this rank)
    for (int c = rank; c < n; c += a.G)
      for (int e = t; e < n; e += kBT) mt.R[e + (i64)c * n] = 0.0;
    int bw = mt.b, bprev = 0;
    bool failed = false;  // a breakdown: the group leaves this matrix
    for (int c0 = 0; c0 < n && alive && !failed;) {
      double* my = slots[phase & 1] + (size_t)rank * kBSlot;
      // ---- the first CholeskyQR's Gram (with the update of step 4 for c0 > 0)
      {
        PassSpec P{};
        P.dst = mt.Q;
        P.ldd = mt.lda;
        P.op2 = 1;
        P.g0 = c0;
        P.gb = bw;
        if (c0 == 0) {
          P.src = oop ? mt.A : mt.Q;
          P.lds = mt.lda;
          P.lo = 0;
          P.hi = oop ? n : bw;
          P.st_lo = 0;
          P.st_hi = oop ? n : 0;
        } else {  // A_{j:k} -= Q_{j-1} Y, Y (bprev x (n - c0)) in M
          P.src = mt.Q;
          P.lds = mt.lda;
          P.lo = c0 - bprev;
          P.hi = n;
          P.st_lo = c0;
          P.st_hi = n;
          P.op1 = 2;
          P.x0u = c0 - bprev;
          P.pu = bprev;
          P.c0u = c0;
          P.qu = n - c0;
          P.Mm = s.M;
        }
        run_pass(P, s, R0, R1, my);
      }
      if (!(alive = group_barrier(a, group, rank, &bar_count, &bar_ok))) break;
      int broken = reduce_cholesky(s, slots[phase & 1], a.G, bw, a.halve != 0, &sh_rej, &sh_broken);
      ++phase;
      while (a.halve && bw > 1 && sh_rej) {  // rejected panel: its Gram again at the narrower width
        bw = halved(bw);
        my = slots[phase & 1] + (size_t)rank * kBSlot;
        PassSpec P{};
        P.src = mt.Q;
        P.lds = mt.lda;
        P.lo = c0;
        P.hi = c0 + bw;
        P.op2 = 1;
        P.g0 = c0;
        P.gb = bw;
        run_pass(P, s, R0, R1, my);
        if (!(alive = group_barrier(a, group, rank, &bar_count, &bar_ok))) break;
        broken = reduce_cholesky(s, slots[phase & 1], a.G, bw, true, &sh_rej, &sh_broken);
        ++phase;
      }
      if (!alive) break;
      if (broken >= 0) {
        if (rank == 0 && t == 0) atomicCAS(&a.status[mi], 0, c0 + broken + 1);
        failed = true;
        break;
      }
      // S1 for the R products (rank 0; read after the next barrier)
      if (rank == 0)
        for (int e = t; e < bw * bw; e += kBT) {
          const int i = e % bw, c = e / bw;
          s1g[e] = i <= c ? su(s, bw, i, c) : 0.0;
        }
      // ---- T1: P = A_j S1^{-1}, then the Gram of P (c0 == 0) or Z = Q_{1:j-1}^T P
      __syncthreads();  // S1 saved from the unscaled factor
      prescale_rows(s, bw);
      {
        my = slots[phase & 1] + (size_t)rank * kBSlot;
        PassSpec P{};
        P.src = mt.Q;
        P.lds = mt.lda;
        P.dst = mt.Q;
        P.ldd = mt.lda;
        P.lo = 0;
        P.hi = c0 + bw;
        P.st_lo = c0;
        P.st_hi = c0 + bw;
        P.op1 = 1;
        P.t0 = c0;
        P.tb = bw;
        if (c0 == 0) {
          P.op2 = 1;
          P.g0 = 0;
          P.gb = bw;
        } else {
          P.op2 = 2;
          P.x0 = 0;
          P.px = c0;
          P.y0 = c0;
          P.qy = bw;
        }
        run_pass(P, s, R0, R1, my);
      }
      if (!(alive = group_barrier(a, group, rank, &bar_count, &bar_ok))) break;
      if (c0 > 0) {
        reduce_tn(s, slots[phase & 1], a.G, c0, bw);  // Z (c0 x bw) in M
        ++phase;
        // ---- RO: P -= Q_{1:j-1} Z, then the Gram of P
        my = slots[phase & 1] + (size_t)rank * kBSlot;
        PassSpec P{};
        P.src = mt.Q;
        P.lds = mt.lda;
        P.dst = mt.Q;
        P.ldd = mt.lda;
        P.lo = 0;
        P.hi = c0 + bw;
        P.st_lo = c0;
        P.st_hi = c0 + bw;
        P.op1 = 2;
        P.x0u = 0;
        P.pu = c0;
        P.c0u = c0;
        P.qu = bw;
        P.Mm = s.M;
        P.op2 = 1;
        P.g0 = c0;
        P.gb = bw;
        run_pass(P, s, R0, R1, my);
        if (!(alive = group_barrier(a, group, rank, &bar_count, &bar_ok))) break;
      }
      broken = reduce_cholesky(s, slots[phase & 1], a.G, bw, false, &sh_rej, &sh_broken);  // S2
      ++phase;
      if (broken >= 0) {
        if (rank == 0 && t == 0) atomicCAS(&a.status[mi], 0, c0 + broken + 1);
        failed = true;
        break;
      }
      // R_jj = S2 S1 and (c0 > 0) R_{1:j-1,j} += Z S1, column slices of this
      // rank; S1's upper triangle staged (packed by columns) in the tile area
      {
        double* s1p = s.tile;
        for (int e = t; e < bw * (bw + 1) / 2; e += kBT) {
          int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
          while ((c + 1) * (c + 2) / 2 <= e) ++c;
          while (c * (c + 1) / 2 > e) --c;
          const int i = e - c * (c + 1) / 2;
          s1p[e] = s1g[(size_t)c * bw + i];
        }
        __syncthreads();
        const int ncol = (bw - rank + a.G - 1) / a.G;  // this rank's columns c = rank + G * k
        const int per = c0 + bw;                       // rows of R above and on the diagonal block
        for (int e = t; e < ncol * per; e += kBT) {
          const int c = rank + a.G * (e / per), r = e % per;
          const double* s1c = s1p + c * (c + 1) / 2;  // S1[0..c][c]
          if (r >= c0) {  // R_jj entry (r - c0, c), on or above the diagonal
            const int rr = r - c0;
            if (rr > c) continue;
            double v = 0.0;
            for (int i = rr; i <= c; ++i) v = fma(su(s, bw, rr, i), s1c[i], v);
            mt.R[(c0 + rr) + (i64)(c0 + c) * n] = v;
          } else {
            double v = mt.R[r + (i64)(c0 + c) * n];
            for (int i = 0; i <= c; ++i) v = fma(s.M[(size_t)r * bw + i], s1c[i], v);
            mt.R[r + (i64)(c0 + c) * n] = v;
          }
        }
        __syncthreads();
      }
      // ---- T2: Q_j = P S2^{-1}, then Y = Q_j^T A_{j+1:k}
      const int wn = n - c0 - bw;
      __syncthreads();  // the R products used the unscaled factor
      prescale_rows(s, bw);
      {
        my = slots[phase & 1] + (size_t)rank * kBSlot;
        PassSpec P{};
        P.src = mt.Q;
        P.lds = mt.lda;
        P.dst = mt.Q;
        P.ldd = mt.lda;
        P.lo = c0;
        P.hi = n;
        P.st_lo = c0;
        P.st_hi = c0 + bw;
        P.op1 = 1;
        P.t0 = c0;
        P.tb = bw;
        if (wn > 0) {
          P.op2 = 2;
          P.x0 = c0;
          P.px = bw;
          P.y0 = c0 + bw;
          P.qy = wn;
        } else {
          P.hi = c0 + bw;
        }
        run_pass(P, s, R0, R1, my);
      }
      if (wn > 0) {
        if (!(alive = group_barrier(a, group, rank, &bar_count, &bar_ok))) break;
        reduce_tn(s, slots[phase & 1], a.G, bw, wn);  // Y (bw x wn) in M
        ++phase;
        for (int c = rank; c < wn; c += a.G)
          for (int r = t; r < bw; r += kBT) mt.R[(c0 + r) + (i64)(c0 + bw + c) * n] = s.M[(size_t)r * wn + c];
      }
      bprev = bw;
      c0 += bw;
    }
    if (!alive) break;
    if (rank == 0 && t == 0) a.bfinal[mi] = bw;
    // the next matrix reuses M, U and the slots only after its first barrier
    __syncthreads();
  }
  if (!alive && rank == 0 && t == 0) {  // this group's unfinished matrices
    for (int k = li; k < l1; ++k) atomicCAS(&a.status[a.order[k]], 0, CQR_STATUS_TIMEOUT);
  }
}

// Copies a parameter blob into the workspace: the descriptor table travels
// as kernel parameters, so a captured graph holds it by value.
constexpr int kBlob = 30000;
struct Blob {
  unsigned char bytes[kBlob];
  int nbytes;
};
__global__ void blob_copy_kernel(const __grid_constant__ Blob blob, unsigned char* dst) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < blob.nbytes; e += gridDim.x * blockDim.x)
    dst[e] = blob.bytes[e];
}

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct BLayout {
  size_t mats, order, gstart, bfinal, part, s1, bar, abort, total;
};

BLayout blayout(int batch, int grid) {
  BLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = a256(off + bytes);
    return o;
  };
  L.mats = take(sizeof(BMat) * (size_t)batch);
  L.order = take(sizeof(int) * (size_t)batch);
  L.gstart = take(sizeof(int) * (size_t)(grid + 1));
  L.bfinal = take(sizeof(int) * (size_t)batch);
  L.part = take(sizeof(double) * 2 * (size_t)grid * kBSlot);
  L.s1 = take(sizeof(double) * (size_t)grid * kBNMax * kBNMax);
  L.bar = take(sizeof(unsigned int) * (size_t)grid);
  L.abort = take(sizeof(int));
  L.total = off;
  return L;
}

int g_grid_cached[64] = {};

int persistent_grid_impl() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return kSMs;
  if (!g_grid_cached[dev]) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = kSMs;
    g_grid_cached[dev] = sms;
  }
  return g_grid_cached[dev];
}

// One-shot test hook (cqr_test_arm_barrier_expiry).
std::mutex g_bhook_mu;
int g_bhook_group = -1, g_bhook_rank = -1, g_bhook_barrier = -1;
unsigned long long g_bhook_ns = 0;

}  // namespace

int batched_persistent_grid() { return persistent_grid_impl(); }

bool batched_persistent_eligible(int batch, const int64_t* m, const int64_t* n, const int* b) {
  for (int i = 0; i < batch; ++i) {
    if (n[i] > kBNMax || n[i] % 4 || b[i] % 4 || b[i] < 4 || n[i] % b[i]) return false;
    if (m[i] < n[i]) return false;
  }
  return true;
}

size_t batched_persistent_workspace(int batch) { return blayout(batch, persistent_grid_impl()).total; }

// Rough device time of one matrix on a group of G CTAs (for the static
// largest-first schedule): its FLOPs at G SMs' FP64 rate, plus per-phase
// costs (barrier, slot sums, the b x b Cholesky on one SM).
static double est_seconds(i64 m, int n, int b, int G) {
  const int k = n / b;
  const double flops = 4.0 * (double)m * n * n;
  const double rate = (double)G * 8.0e9;
  const double chol = (double)b * b * b / 6.0 / 4.0e9 + 4e-6;
  return flops / rate + (4.0 * k) * (6e-6 + chol);
}

cudaError_t batched_persistent_run(int batch, const int64_t* m, const int64_t* n, const int64_t* lda,
                                   const int* b, double* const* A, double* const* Q, double* const* R,
                                   int* status, void* workspace, int G, bool halve, cudaStream_t st) {
  const int grid = persistent_grid_impl();
  if (G < 1 || grid % G) return cudaErrorInvalidValue;
  const int groups = grid / G;
  const BLayout L = blayout(batch, grid);
  char* ws = (char*)workspace;
  // descriptors and the static schedule (largest estimated time first, each
  // to the group with the least work so far)
  std::vector<BMat> mats((size_t)batch);
  int nmax = 4, bmax = 4;
  std::vector<std::pair<double, int>> by;
  for (int i = 0; i < batch; ++i) {
    mats[i].A = A[i];
    mats[i].Q = Q[i];
    mats[i].R = R[i];
    mats[i].m = m[i];
    mats[i].lda = lda[i];
    mats[i].n = (int)n[i];
    mats[i].b = b[i];
    nmax = std::max(nmax, (int)n[i]);
    bmax = std::max(bmax, b[i]);
    by.push_back({est_seconds(m[i], (int)n[i], b[i], G), i});
  }
  std::stable_sort(by.begin(), by.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
    return x.first > y.first;
  });
  std::vector<double> load((size_t)groups, 0.0);
  std::vector<std::vector<int>> lists((size_t)groups);
  for (const auto& e : by) {
    int g = 0;
    for (int h = 1; h < groups; ++h)
      if (load[h] < load[g]) g = h;
    load[g] += e.first;
    lists[g].push_back(e.second);
  }
  std::vector<int> order, gstart((size_t)grid + 1, batch);
  for (int g = 0; g < groups; ++g) {
    gstart[g] = (int)order.size();
    for (int i : lists[g]) order.push_back(i);
  }
  for (int g = groups; g <= grid; ++g) gstart[g] = batch;
  // descriptor table, schedule: kernel-parameter blobs into the workspace
  auto upload = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    const unsigned char* p = (const unsigned char*)src;
    for (size_t done = 0; done < bytes; done += kBlob) {
      Blob blob;
      blob.nbytes = (int)std::min((size_t)kBlob, bytes - done);
      memcpy(blob.bytes, p + done, (size_t)blob.nbytes);
      prof_begin(kMisc, st);
      blob_copy_kernel<<<8, 256, 0, st>>>(blob, (unsigned char*)ws + off + done);
      prof_end(kMisc, 0.0, st);
      TRY_RET(cudaGetLastError());
    }
    return cudaSuccess;
  };
  if (batch > 0) {
    TRY_RET(upload(L.mats, mats.data(), sizeof(BMat) * (size_t)batch));
    TRY_RET(upload(L.order, order.data(), sizeof(int) * (size_t)batch));
  }
  TRY_RET(upload(L.gstart, gstart.data(), sizeof(int) * ((size_t)grid + 1)));
  TRY_RET(cudaMemsetAsync(ws + L.bar, 0, sizeof(unsigned int) * (size_t)grid, st));
  TRY_RET(cudaMemsetAsync(ws + L.abort, 0, sizeof(int), st));
  TRY_RET(cudaMemsetAsync(status, 0, sizeof(int) * (size_t)batch, st));
  BArgs a{};
  a.mats = (const BMat*)(ws + L.mats);
  a.order = (const int*)(ws + L.order);
  a.gstart = (const int*)(ws + L.gstart);
  a.status = status;
  a.bfinal = (int*)(ws + L.bfinal);
  a.part = (double*)(ws + L.part);
  a.s1 = (double*)(ws + L.s1);
  a.bar = (unsigned int*)(ws + L.bar);
  a.abort = (int*)(ws + L.abort);
  a.G = G;
  a.nmax = nmax;
  a.bmax = bmax;
  a.halve = halve ? 1 : 0;
  a.wait_ns = kBWaitNs;
  a.hook_group = a.hook_rank = a.hook_barrier = -1;
  {
    std::lock_guard<std::mutex> lk(g_bhook_mu);
    if (g_bhook_group >= 0) {
      a.hook_group = g_bhook_group;
      a.hook_rank = g_bhook_rank;
      a.hook_barrier = g_bhook_barrier;
      a.wait_ns = g_bhook_ns;
      g_bhook_group = -1;
    }
  }
  const size_t smem = bsmem_bytes(nmax, bmax);
  TRY_RET(cudaFuncSetAttribute(batched_mcqr2gs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  TRY_RET(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_mcqr2gs_kernel, kBT, smem));
  if (occ < 1) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  double flops = 0.0;
  for (int i = 0; i < batch; ++i) flops += 4.0 * (double)m[i] * n[i] * n[i];
  prof_begin(kBatched, st);
  cudaError_t e = cudaLaunchKernelEx(&cfg, batched_mcqr2gs_kernel, a);
  prof_end(kBatched, flops, st);
  return e;
}

cudaError_t batched_persistent_panels(int batch, const void* workspace, int* host_b, cudaStream_t st) {
  const BLayout L = blayout(batch, persistent_grid_impl());
  TRY_RET(cudaMemcpyAsync(host_b, (const char*)workspace + L.bfinal, sizeof(int) * (size_t)batch,
                          cudaMemcpyDeviceToHost, st));
  return cudaStreamSynchronize(st);
}

}  // namespace cqr

extern "C" int cqr_test_arm_barrier_expiry(int group, int rank, int barrier, long long wait_ns) {
  if (group < -1) return -1;
  std::lock_guard<std::mutex> lk(cqr::g_bhook_mu);
  if (group == -1) {
    cqr::g_bhook_group = -1;
    return 0;
  }
  if (rank < 0) return -2;
  if (barrier < 1) return -3;
  if (wait_ns < 1 || wait_ns > (long long)cqr::kBWaitNs) return -4;
  cqr::g_bhook_group = group;
  cqr::g_bhook_rank = rank;
  cqr::g_bhook_barrier = barrier;
  cqr::g_bhook_ns = (unsigned long long)wait_ns;
  return 0;
}
