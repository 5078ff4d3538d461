// FP64 peak microbenchmarks: the denominators of the roofline fractions the
// library reports.  Three probes, each a single-wave grid of independent
// multiply-add chains on every SM:
//   kind 0  DFMA on the CUDA cores: each thread runs kDfmaChains independent
//           fused multiply-add chains on register operands;
//   kind 1  FP64 tensor cores, mma.sync.aligned.m8n8k4 .f64 (512 flop per
//           warp instruction): kMmaChains independent accumulators per warp;
//   kind 2  FP64 tensor cores, mma.sync.aligned.m16n8k16 .f64 (4096 flop per
//           warp instruction), likewise.
// Every block records its SM id and the SM clock counter (clock64) at its
// start and end.  Per SM, the flops of its blocks divided by the cycles from
// its first start to its last end give flop/clk/SM, a figure that does not
// depend on the clock the GPU ran at; the CUDA-event time of the launch
// gives GFLOP/s, and cycles / time the effective SM clock.
#include "cqr_common.cuh"

namespace cqr {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kDfmaChains = 12;
constexpr int kMmaChains = 4;

__device__ double g_probe_sink;

struct BlockClock {
  long long start, end;
  int sm;
};

// Per-block clock records (module data, so the probe allocates nothing).
constexpr int kMaxProbeBlocks = 4096;
__device__ BlockClock g_probe_rec[kMaxProbeBlocks];

__device__ __forceinline__ int sm_id() {
  int s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

__device__ __forceinline__ void record_start(BlockClock* rec, long long& t0) {
  __syncthreads();
  t0 = clock64();
}
__device__ __forceinline__ void record_end(BlockClock* rec, long long t0) {
  __syncthreads();
  if (threadIdx.x == 0) {
    rec[blockIdx.x].start = t0;
    rec[blockIdx.x].end = clock64();
    rec[blockIdx.x].sm = sm_id();
  }
}

__global__ void __launch_bounds__(kProbeThreads) dfma_probe_kernel(int iters, BlockClock* rec) {
  // operands in registers, derived from the thread index so nothing folds
  const double x = 1.0 - 1e-9 * (double)(threadIdx.x & 7);
  const double y = 1e-12 * (double)(threadIdx.x + 1);
  double acc[kDfmaChains];
#pragma unroll
  for (int i = 0; i < kDfmaChains; ++i) acc[i] = threadIdx.x * 1e-3 + i;
  long long t0;
  record_start(rec, t0);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < kDfmaChains; ++i) acc[i] = fma(acc[i], x, y);
  record_end(rec, t0);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kDfmaChains; ++i) s += acc[i];
  if (s == 1.2345e-300) g_probe_sink = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) dmma_m8n8k4_probe_kernel(int iters, BlockClock* rec) {
  const double a = 1.0 - 1e-9 * (double)(threadIdx.x & 7);
  const double b = 1e-12 * (double)(threadIdx.x + 1);
  double d[kMmaChains][2];
#pragma unroll
  for (int i = 0; i < kMmaChains; ++i) d[i][0] = d[i][1] = threadIdx.x * 1e-3 + i;
  long long t0;
  record_start(rec, t0);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < kMmaChains; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(d[i][0]), "+d"(d[i][1])
                   : "d"(a), "d"(b));
  record_end(rec, t0);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kMmaChains; ++i) s += d[i][0] + d[i][1];
  if (s == 1.2345e-300) g_probe_sink = s;
}

__global__ void __launch_bounds__(kProbeThreads) dmma_m16n8k16_probe_kernel(int iters, BlockClock* rec) {
  double a[8], b[4];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = 1.0 - 1e-9 * (double)((threadIdx.x + i) & 7);
#pragma unroll
  for (int i = 0; i < 4; ++i) b[i] = 1e-12 * (double)(threadIdx.x + 1 + i);
  double d[kMmaChains][4];
#pragma unroll
  for (int i = 0; i < kMmaChains; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) d[i][j] = threadIdx.x * 1e-3 + i + j;
  long long t0;
  record_start(rec, t0);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < kMmaChains; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, "
          "{%12,%13,%14,%15}, {%0,%1,%2,%3};"
          : "+d"(d[i][0]), "+d"(d[i][1]), "+d"(d[i][2]), "+d"(d[i][3])
          : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]), "d"(b[0]),
            "d"(b[1]), "d"(b[2]), "d"(b[3]));
  record_end(rec, t0);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kMmaChains; ++i) s += d[i][0] + d[i][1] + d[i][2] + d[i][3];
  if (s == 1.2345e-300) g_probe_sink = s;
}

// FLOPs one block performs in `iters` iterations.
double block_flops(int kind, int iters) {
  const double warps = kProbeThreads / 32;
  switch (kind) {
    case 0: return 2.0 * kDfmaChains * (double)iters * kProbeThreads;
    case 1: return 2.0 * 8 * 8 * 4 * kMmaChains * (double)iters * warps;
    default: return 2.0 * 16 * 8 * 16 * kMmaChains * (double)iters * warps;
  }
}

cudaError_t launch_probe(int kind, int blocks, int iters, BlockClock* rec, cudaStream_t st) {
  prof_begin(kMisc, st);
  switch (kind) {
    case 0: dfma_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(iters, rec); break;
    case 1: dmma_m8n8k4_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(iters, rec); break;
    default: dmma_m16n8k16_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(iters, rec); break;
  }
  prof_end(kMisc, 0.0, st);
  return cudaGetLastError();
}

int resident_blocks(int kind) {
  int occ = 0;
  switch (kind) {
    case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dfma_probe_kernel, kProbeThreads, 0); break;
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dmma_m8n8k4_probe_kernel, kProbeThreads, 0); break;
    default:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dmma_m16n8k16_probe_kernel, kProbeThreads, 0);
      break;
  }
  return occ > 0 ? occ : 1;
}

}  // namespace

int probe_fp64(int kind, int iters, double* gflops, double* flop_per_clk_sm, double* sm_mhz) {
  if (kind < 0 || kind > 2 || iters < 1) return -1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -2;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return -2;
  // one wave: every block resident from the start
  const int per_sm = resident_blocks(kind) < 4 ? resident_blocks(kind) : 4;
  const int blocks = sms * per_sm;
  if (blocks > kMaxProbeBlocks) return -2;
  BlockClock* rec = nullptr;
  if (cudaGetSymbolAddress((void**)&rec, g_probe_rec) != cudaSuccess || !rec) return -2;
  BlockClock* h = new BlockClock[blocks];
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t err = cudaSuccess;
  // warm-up: clocks settle, then three timed launches, the fastest kept
  for (int w = 0; w < 2 && err == cudaSuccess; ++w) err = launch_probe(kind, blocks, iters, rec, 0);
  float best_ms = 0.f;
  double best_fpc = 0.0;
  long long best_cycles = 0;
  for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
    cudaEventRecord(e0, 0);
    err = launch_probe(kind, blocks, iters, rec, 0);
    cudaEventRecord(e1, 0);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    err = cudaMemcpy(h, rec, sizeof(BlockClock) * blocks, cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) break;
    // per SM: first start to last end
    double fpc_sum = 0.0;
    long long cyc_max = 0;
    int used = 0;
    for (int s = 0; s < sms; ++s) {
      long long lo = 0, hi = 0;
      int nb = 0;
      for (int b = 0; b < blocks; ++b) {
        if (h[b].sm != s) continue;
        if (nb == 0 || h[b].start < lo) lo = h[b].start;
        if (nb == 0 || h[b].end > hi) hi = h[b].end;
        ++nb;
      }
      if (nb == 0 || hi <= lo) continue;
      fpc_sum += block_flops(kind, iters) * nb / (double)(hi - lo);
      if (hi - lo > cyc_max) cyc_max = hi - lo;
      ++used;
    }
    if (used == 0) {
      err = cudaErrorUnknown;
      break;
    }
    const double fpc = fpc_sum / used;
    if (ms > 0.f && (best_ms == 0.f || ms < best_ms)) {
      best_ms = ms;
      best_fpc = fpc;
      best_cycles = cyc_max;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  delete[] h;
  if (err != cudaSuccess || best_ms <= 0.f) return -3;
  const double flops = block_flops(kind, iters) * blocks;
  if (gflops) *gflops = flops / (best_ms * 1e-3) / 1e9;
  if (flop_per_clk_sm) *flop_per_clk_sm = best_fpc;
  if (sm_mhz) *sm_mhz = (double)best_cycles / (best_ms * 1e-3) / 1e6;
  return 0;
}

}  // namespace cqr
