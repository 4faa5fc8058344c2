// Cholesky factorisation that needs no caller-provided workspace and allocates nothing.
//
// Some callers cannot hand the library device scratch: a host application whose
// device memory is owned by another allocator (a framework's caching pool, a
// serving runtime with a fixed memory plan) may not be allowed to call cudaMalloc
// behind that allocator's back, and code on a latency-critical path may not accept
// the implicit device-wide synchronisation a cudaMalloc/cudaFree can cause.  For
// them, qdwhp_potrf_f64_noalloc runs the same factorisation as qdwhp_potrf_f64 but
// takes its scratch from a fixed array in the library's own device memory.
//
// The array is a file-scope __device__ variable, so every GPU that loads the library
// keeps its kNoallocBytes until the process exits.  Host code cannot use the
// array's name as a device address (on the host it names a stand-in object), so the
// device address is looked up with cudaGetSymbolAddress once per device, with that
// device current, the first time the entry point runs there.
#include <mutex>

#include "internal.h"

namespace qdwhp {

namespace {

constexpr int64_t kNoallocMaxN = QDWHP_POTRF_NOALLOC_MAX_N;
// Leaf inverses (ceil(n / 64) blocks of 64 x 64) + the triangular-solve buffer (n x 64)
// + the failure flag, for n up to kNoallocMaxN.
constexpr size_t kNoallocLinvElems = (size_t)((kNoallocMaxN + kCholNB - 1) / kCholNB) * kCholNB * kCholNB;
constexpr size_t kNoallocScratchElems = (size_t)kNoallocMaxN * kCholNB;
constexpr size_t kNoallocElems = kNoallocLinvElems + kNoallocScratchElems + 32;   // 4 MB in total

static __device__ __align__(256) double g_noalloc_scratch[kNoallocElems];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
qdwhp_status noalloc_scratch(double** out) {
  int dev = 0;
  QDWHP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return QDWHP_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    QDWHP_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return QDWHP_OK;
}

}  // namespace

}  // namespace qdwhp

using namespace qdwhp;

extern "C" {

QDWHP_API qdwhp_status qdwhp_potrf_f64_noalloc(int64_t n, double* Z, int64_t ldz, int* info_host, void* stream) {
  if (info_host) *info_host = 0;
  if (n < 0 || (n > 0 && (Z == nullptr || ldz < n))) return QDWHP_ERR_ARG;
  if (n > kNoallocMaxN) {
    set_error_message("qdwhp_potrf_f64_noalloc: n exceeds the static scratch limit of 4096");
    return QDWHP_ERR_ARG;
  }
  if (n == 0) return QDWHP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  double* base = nullptr;
  QDWHP_TRY(noalloc_scratch(&base));
  double* Linv = base;
  double* scratch = base + kNoallocLinvElems;
  int* fail = reinterpret_cast<int*>(base + kNoallocLinvElems + kNoallocScratchElems);
  // The array keeps the previous call's contents: the failure flag must start at zero.
  QDWHP_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int), st));
  QDWHP_TRY(potrf(st, n, Z, ldz, Linv, scratch, fail));
  int h = 0;
  QDWHP_CUDA_TRY(cudaMemcpyAsync(&h, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
  QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  if (info_host) *info_host = h;
  return h ? QDWHP_ERR_BREAKDOWN : QDWHP_OK;
}

}  // extern "C"
