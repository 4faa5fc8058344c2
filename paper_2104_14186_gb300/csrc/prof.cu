// Launch counting and opt-in timing of the DMMA GEMM launches.
//
// Timing places a CUDA event pair around every GEMM (and its split-K reduction) on
// the stream it is launched on, and sums the pairs' elapsed times when profiling
// ends, so callers can report the achieved FP64 rate of the dominant kernel from
// inside a real solve.  Profiling is process-wide and meant for one host thread.
#include <atomic>
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
std::mutex g_coop_mu;
cudaEvent_t g_coop_last = nullptr;
}  // namespace

qdwhp_status launch_cooperative(const void* fn, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t st) {
  // Cooperative kernels run one at a time on the GPU: each waits (on its own stream) for the
  // previous one, so two grids never hold parts of the GPU while waiting at their barriers.
  std::lock_guard<std::mutex> lk(g_coop_mu);
  if (g_coop_last == nullptr) QDWHP_CUDA_TRY(cudaEventCreateWithFlags(&g_coop_last, cudaEventDisableTiming));
  else QDWHP_CUDA_TRY(cudaStreamWaitEvent(st, g_coop_last, 0));
  QDWHP_CUDA_TRY(cudaLaunchCooperativeKernel(fn, grid, block, args, smem, st));
  QDWHP_LAUNCH_CHECK();
  QDWHP_CUDA_TRY(cudaEventRecord(g_coop_last, st));
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
