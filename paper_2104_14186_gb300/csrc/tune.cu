// Run-time launch parameters per size class, set by the autotuner (or left at their
// defaults).  Each knob picks between launch shapes that compute the same result:
//   kTunePanelRows     rows per CTA of the cooperative Householder panel (its CTA count is
//                      ceil(R / rows), at most 96), by the panel's row count R;
//   kTuneJacobiWarps   least warps (pairs) per CTA of a cooperative Jacobi sweep, by the
//                      column count (fewer, fuller CTAs meet at a cheaper grid barrier);
//   kTuneSplitkPerSM   CTAs per SM that split-K aims for when a product has few output
//                      tiles, by max(m, n).
// Size classes: <= 128, <= 256, <= 512, <= 1024, larger.  The bounds keep every launch
// valid: panel shared memory stays <= 128 KB, a sweep's grid never exceeds the SM count.
#include <atomic>

#include "internal.h"

namespace qdwhp {

namespace {

constexpr int kDefaults[kTuneKnobs] = {64, 2, 2};
constexpr int kLow[kTuneKnobs] = {16, 1, 1};
constexpr int kHigh[kTuneKnobs] = {512, 16, 8};

std::atomic<int> g_tune[kTuneKnobs][kTuneClasses] = {
    {{64}, {64}, {64}, {64}, {64}},
    {{2}, {2}, {2}, {2}, {2}},
    {{2}, {2}, {2}, {2}, {2}},
};

}  // namespace

int tune_class(int64_t size) {
  if (size <= 128) return 0;
  if (size <= 256) return 1;
  if (size <= 512) return 2;
  if (size <= 1024) return 3;
  return 4;
}

int tune_value(TuneKnob knob, int64_t size) {
  return g_tune[knob][tune_class(size)].load(std::memory_order_relaxed);
}

}  // namespace qdwhp

using namespace qdwhp;

extern "C" {

QDWHP_API qdwhp_status qdwhp_tune_set(int32_t knob, int32_t size_class, int32_t value) {
  if (knob < 0 || knob >= kTuneKnobs || size_class < 0 || size_class >= kTuneClasses) return QDWHP_ERR_ARG;
  if (value < kLow[knob] || value > kHigh[knob]) return QDWHP_ERR_ARG;
  g_tune[knob][size_class].store(value, std::memory_order_relaxed);
  return QDWHP_OK;
}

QDWHP_API int32_t qdwhp_tune_get(int32_t knob, int32_t size_class) {
  if (knob < 0 || knob >= kTuneKnobs || size_class < 0 || size_class >= kTuneClasses) return -1;
  return g_tune[knob][size_class].load(std::memory_order_relaxed);
}

QDWHP_API void qdwhp_tune_reset(void) {
  for (int k = 0; k < kTuneKnobs; ++k)
    for (int c = 0; c < kTuneClasses; ++c) g_tune[k][c].store(kDefaults[k], std::memory_order_relaxed);
}

}  // extern "C"
