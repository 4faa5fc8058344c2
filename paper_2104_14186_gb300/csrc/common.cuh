// Shared device/host helpers of the qdwhp library (internal).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <cmath>
#include <algorithm>
#include <cstring>

#include "../../include/qdwhp.h"

namespace qdwhp {

constexpr int kNumSMs = 152;          // GB300: 2 dies x 76 SMs (queried at run time where it matters)

#define QDWHP_CUDA_TRY(expr)                                   \
  do {                                                          \
    cudaError_t _e = (expr);                                    \
    if (_e != cudaSuccess) {                                    \
      ::qdwhp::set_last_error(_e, #expr, __FILE__, __LINE__);   \
      return QDWHP_ERR_CUDA;                                    \
    }                                                           \
  } while (0)

#define QDWHP_TRY(expr)                       \
  do {                                         \
    qdwhp_status _s = (expr);                  \
    if (_s != QDWHP_OK) return _s;             \
  } while (0)

// Every kernel launch is followed by exactly one QDWHP_LAUNCH_CHECK(), which also
// counts it (qdwhp_launch_count()).
#define QDWHP_LAUNCH_CHECK()                 \
  do {                                       \
    ::qdwhp::note_launch();                  \
    QDWHP_CUDA_TRY(cudaGetLastError());      \
  } while (0)

void set_last_error(cudaError_t e, const char* what, const char* file, int line);
// Sets the text returned by qdwhp_last_error_message() for a non-CUDA error.
void set_error_message(const char* msg);
void note_launch();
// Launches a cooperative kernel behind the process-wide gate that keeps the CTAs of all
// cooperative kernels that can be in flight together at most the SM count (streams of
// concurrent solves may otherwise oversubscribe the GPU with grids waiting at barriers).
qdwhp_status launch_cooperative(const void* fn, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t st);

// Opt-in timing of the DMMA GEMM launches (CUDA events around each launch on its stream).
bool gemm_prof_enabled();
// Records the start event; returns a slot id for gemm_prof_end (or -1 when disabled).
int gemm_prof_start(cudaStream_t st, double flops, const double* shape);
void gemm_prof_stop(cudaStream_t st, int slot);

// Device-side error flags written by kernels (bitwise OR into ws->flags).
enum DeviceFlag : unsigned {
  FLAG_NONFINITE = 1u,
  FLAG_BREAKDOWN = 2u,   // non-positive pivot in a Cholesky leaf
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum; every thread gets the result.  `red` must hold >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) {
    t = warp_sum(t);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a counter-based generator:
// output i of stream `seed` is the finaliser of seed + (i + 1) * golden.
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Uniform double in [-1, 1) from the top 53 bits (exact in binary64).
__host__ __device__ __forceinline__ double uniform_pm1_at(uint64_t seed, uint64_t i) {
  return 2.0 * (double)(splitmix64_at(seed, i) >> 11) * 0x1.0p-53 - 1.0;
}

constexpr uint64_t kStreamLanczos = 0x4C414E43ull;   // "LANC"
constexpr uint64_t kStreamBlock = 0x424C4F43ull;     // "BLOC"
constexpr uint64_t kStreamOmega = 0x4F4D4547ull;     // "OMEG"

// Bump allocator over a caller-owned device workspace.  Every carve is 256-byte aligned.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  bool dry = false;           // sizing pass: count bytes, hand out nothing
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    size_t off = used;
    used += bytes;
    if (dry || base == nullptr || used > cap) return nullptr;
    return reinterpret_cast<T*>(base + off);
  }
  bool ok() const { return dry || (base != nullptr && used <= cap); }
};

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace qdwhp
