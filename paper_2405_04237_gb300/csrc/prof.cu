// Launch accounting and optional per-launch timing.
//
// Every kernel launch of the library passes through prof_begin/prof_end.
// The launch counter is always kept.  When timing is enabled, each launch
// is bracketed by two CUDA events recorded on its own stream and tagged with
// its kernel class and the algorithmic FLOP count of the work it performs,
// so a caller can state achieved FLOP/s per kernel class against the FP64
// roofline.  Timing is off by default (events inside a stream capture would
// become graph nodes; the factorisation itself never needs them).
#include <atomic>
#include <mutex>
#include <vector>

#include "cqr.h"
#include "cqr_common.cuh"

namespace cqr {

namespace {

struct Rec {
  int cls;
  double flops;
  cudaEvent_t e0, e1;
};

std::atomic<unsigned long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
size_t g_cap = 0;
thread_local int t_open = -1;

const char* kNames[kNumClasses] = {"gram_syrk", "projection_tn", "split_reduce", "cholesky", "trsm", "update_gemm",
                                   "misc", "batched"};

}  // namespace

void prof_begin(int cls, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  t_open = -1;
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_recs.size() >= g_cap) return;
  Rec r;
  r.cls = cls;
  r.flops = 0.0;
  r.e0 = g_pool[2 * g_recs.size()];
  r.e1 = g_pool[2 * g_recs.size() + 1];
  cudaEventRecord(r.e0, st);
  g_recs.push_back(r);
  t_open = (int)g_recs.size() - 1;
}

void prof_end(int cls, double flops, cudaStream_t st) {
  (void)cls;
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (t_open < 0 || t_open >= (int)g_recs.size()) return;
  g_recs[t_open].flops = flops;
  cudaEventRecord(g_recs[t_open].e1, st);
  t_open = -1;
}

}  // namespace cqr

using namespace cqr;

extern "C" {

unsigned long long cqr_launch_count(void) { return g_launches.load(); }

int cqr_profile_enable(int capacity) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (capacity < 1) return -1;
  if ((size_t)capacity > g_cap) {
    for (size_t i = g_pool.size(); i < 2 * (size_t)capacity; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return CQR_ERR_CUDA;
      g_pool.push_back(e);
    }
    g_cap = (size_t)capacity;
  }
  g_recs.clear();
  g_on = true;
  return 0;
}

int cqr_profile_disable(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = false;
  return 0;
}

int cqr_profile_read(int cls, long long* launches, double* total_ms, double* flops) {
  if (cls < 0 || cls >= kNumClasses || !launches || !total_ms || !flops) return -1;
  std::lock_guard<std::mutex> lk(g_mu);
  long long n = 0;
  double ms = 0.0, fl = 0.0;
  for (const Rec& r : g_recs) {
    if (r.cls != cls) continue;
    if (cudaEventSynchronize(r.e1) != cudaSuccess) return CQR_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.e0, r.e1) != cudaSuccess) return CQR_ERR_CUDA;
    ++n;
    ms += t;
    fl += r.flops;
  }
  *launches = n;
  *total_ms = ms;
  *flops = fl;
  return 0;
}

const char* cqr_kernel_class_name(int cls) {
  if (cls < 0 || cls >= kNumClasses) return "unknown";
  return kNames[cls];
}

}  // extern "C"
