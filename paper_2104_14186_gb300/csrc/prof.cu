// Launch counting and opt-in timing of the DMMA GEMM launches.
//
// Timing places a CUDA event pair around every GEMM (and its split-K reduction) on
// the stream it is launched on, and sums the pairs' elapsed times when profiling
// ends, so callers can report the achieved FP64 rate of the dominant kernel from
// inside a real solve.  Profiling is process-wide and meant for one host thread.
#include <atomic>
#include <deque>
#include <mutex>
#include <vector>

#include "internal.h"

namespace qdwhp {

namespace {
std::atomic<unsigned long long> g_launches{0};
struct ProfSlot {
  cudaEvent_t a = nullptr, b = nullptr;
  double flops = 0.0;
  double shape[5] = {0, 0, 0, 0, 0};   // m, n, k, lower, split
};
std::vector<double> g_records;          // 6 doubles per GEMM of the last profile: m, n, k, lower, split, ms
std::mutex g_mu;
bool g_on = false;
std::vector<ProfSlot> g_slots;
size_t g_used = 0;
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
// In-flight cooperative kernels: their completion events and CTA counts, oldest first.
struct CoopEntry {
  cudaEvent_t done;
  int ctas;
};
std::mutex g_coop_mu;
std::deque<CoopEntry> g_coop_inflight;
std::vector<cudaEvent_t> g_coop_free_events;
int g_coop_total = 0;
int g_coop_capacity = 0;
}  // namespace

qdwhp_status launch_cooperative(const void* fn, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t st) {
  // Cooperative kernels may run concurrently (streams of concurrent solves) as long as the CTAs
  // of all cooperative grids that can be in flight together number at most the SM count: each
  // CTA fits on an empty SM and ordinary kernels always drain, so every such grid eventually
  // becomes fully resident and its grid barriers complete.  Before a launch that would exceed
  // the budget, the stream waits (on the GPU) for the oldest in-flight cooperative kernels.
  std::lock_guard<std::mutex> lk(g_coop_mu);
  if (g_coop_capacity == 0) {
    int dev = 0, sms = kNumSMs;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_coop_capacity = sms;
  }
  const int ctas = (int)(grid.x * grid.y * grid.z);
  if (ctas > g_coop_capacity) return QDWHP_ERR_ARG;
  // forget kernels that have finished
  while (!g_coop_inflight.empty() && cudaEventQuery(g_coop_inflight.front().done) == cudaSuccess) {
    g_coop_total -= g_coop_inflight.front().ctas;
    g_coop_free_events.push_back(g_coop_inflight.front().done);
    g_coop_inflight.pop_front();
  }
  cudaGetLastError();   // cudaEventQuery reports cudaErrorNotReady for running kernels
  while (g_coop_total + ctas > g_coop_capacity && !g_coop_inflight.empty()) {
    QDWHP_CUDA_TRY(cudaStreamWaitEvent(st, g_coop_inflight.front().done, 0));
    g_coop_total -= g_coop_inflight.front().ctas;
    g_coop_free_events.push_back(g_coop_inflight.front().done);
    g_coop_inflight.pop_front();
  }
  QDWHP_CUDA_TRY(cudaLaunchCooperativeKernel(fn, grid, block, args, smem, st));
  QDWHP_LAUNCH_CHECK();
  cudaEvent_t ev = nullptr;
  if (!g_coop_free_events.empty()) {
    ev = g_coop_free_events.back();
    g_coop_free_events.pop_back();
  } else {
    QDWHP_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  QDWHP_CUDA_TRY(cudaEventRecord(ev, st));
  g_coop_inflight.push_back({ev, ctas});
  g_coop_total += ctas;
  return QDWHP_OK;
}

bool gemm_prof_enabled() { return g_on; }

int gemm_prof_start(cudaStream_t st, double flops, const double* shape) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return -1;
  if (g_used == g_slots.size()) {
    ProfSlot s;
    if (cudaEventCreate(&s.a) != cudaSuccess || cudaEventCreate(&s.b) != cudaSuccess) return -1;
    g_slots.push_back(s);
  }
  const int slot = (int)g_used++;
  g_slots[slot].flops = flops;
  for (int i = 0; i < 5; ++i) g_slots[slot].shape[i] = shape ? shape[i] : 0.0;
  cudaEventRecord(g_slots[slot].a, st);
  return slot;
}

void gemm_prof_stop(cudaStream_t st, int slot) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (slot >= 0 && (size_t)slot < g_used) cudaEventRecord(g_slots[slot].b, st);
}

}  // namespace qdwhp

using namespace qdwhp;

extern "C" {

QDWHP_API unsigned long long qdwhp_launch_count(void) { return g_launches.load(); }

QDWHP_API qdwhp_status qdwhp_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = true;
  g_used = 0;
  return QDWHP_OK;
}

QDWHP_API qdwhp_status qdwhp_profile_end(double* gemm_ms, double* gemm_flops, int64_t* gemm_launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = false;
  double ms_total = 0.0, fl = 0.0;
  g_records.clear();
  for (size_t i = 0; i < g_used; ++i) {
    QDWHP_CUDA_TRY(cudaEventSynchronize(g_slots[i].b));
    float ms = 0.f;
    QDWHP_CUDA_TRY(cudaEventElapsedTime(&ms, g_slots[i].a, g_slots[i].b));
    ms_total += ms;
    fl += g_slots[i].flops;
    for (int j = 0; j < 5; ++j) g_records.push_back(g_slots[i].shape[j]);
    g_records.push_back(ms);
  }
  if (gemm_ms) *gemm_ms = ms_total;
  if (gemm_flops) *gemm_flops = fl;
  if (gemm_launches) *gemm_launches = (int64_t)g_used;
  g_used = 0;
  return QDWHP_OK;
}

QDWHP_API int64_t qdwhp_profile_records(double* out, int64_t capacity) {
  std::lock_guard<std::mutex> lk(g_mu);
  const int64_t n = (int64_t)g_records.size() / 6;
  if (out != nullptr)
    for (int64_t i = 0; i < std::min(n, capacity) * 6; ++i) out[i] = g_records[i];
  return n;
}

}  // extern "C"
