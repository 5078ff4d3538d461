// Launch accounting and optional per-launch timing.
//
// Every kernel launch of the library passes through prof_begin/prof_end.
// The launch counter is always kept.  When timing is enabled, each launch
// is bracketed by two CUDA events recorded on its own stream and tagged with
// its kernel class and the algorithmic FLOP count of the work it performs,
// so a caller can state achieved FLOP/s per kernel class against the FP64
// roofline.  Timing is off by default (events inside a stream capture would
// become graph nodes; the factorisation itself never needs them).
#include <nvtx3/nvToolsExt.h>
#include <stdio.h>

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

// Phase tracing: NVTX (a no-op unless a tool is attached) plus an optional
// caller callback.
std::mutex g_trace_mu;
cqr_trace_fn g_trace = nullptr;
void* g_trace_ctx = nullptr;

nvtxDomainHandle_t trace_domain() {
  static nvtxDomainHandle_t d = nvtxDomainCreateA("cqr");
  return d;
}

void trace_emit(const char* name, int panel, int begin) {
  cqr_trace_fn fn;
  void* ctx;
  {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    fn = g_trace;
    ctx = g_trace_ctx;
  }
  if (fn) fn(name, panel, begin, ctx);
}

}  // namespace

TracePhase::TracePhase(const char* n, int p) : name(n), panel(p) {
  char msg[64];
  if (panel >= 0)
    snprintf(msg, sizeof msg, "%s %d", name, panel);
  else
    snprintf(msg, sizeof msg, "%s", name);
  nvtxEventAttributes_t at = {};
  at.version = NVTX_VERSION;
  at.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
  at.messageType = NVTX_MESSAGE_TYPE_ASCII;
  at.message.ascii = msg;
  nvtxDomainRangePushEx(trace_domain(), &at);
  trace_emit(name, panel, 1);
}

TracePhase::~TracePhase() {
  trace_emit(name, panel, 0);
  nvtxDomainRangePop(trace_domain());
}

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

int cqr_set_trace(cqr_trace_fn fn, void* ctx) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace = fn;
  g_trace_ctx = fn ? ctx : nullptr;
  return 0;
}

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
