// Internal host-side interfaces shared by the library's translation units.
#pragma once

#include <atomic>
#include <mutex>

#include "common.cuh"

namespace qdwhp {

// Runs a setter once per device, the first time that device is current, and again on a later
// call if it failed.  Function attributes (cudaFuncSetAttribute) and __constant__ tables act on
// the current device only, so a process-wide once would leave a second device unconfigured.
class PerDeviceOnce {
 public:
  template <class F>
  cudaError_t run(F&& set) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return set();
    if (done_[dev].load(std::memory_order_acquire)) return cudaSuccess;   // every later launch: no lock
    std::lock_guard<std::mutex> lk(mu_);
    if (done_[dev].load(std::memory_order_relaxed)) return cudaSuccess;
    e = set();
    if (e == cudaSuccess) done_[dev].store(true, std::memory_order_release);
    return e;
  }

 private:
  static constexpr int kMaxDevices = 64;
  std::mutex mu_;
  std::atomic<bool> done_[kMaxDevices] = {};
};

enum Uplo { FULL = 0, LOWER = 1 };

// ---- tune.cu ----
// Run-time launch parameters per size class (<= 128, <= 256, <= 512, <= 1024, larger),
// set through qdwhp_tune_set by the autotuner.
enum TuneKnob { kTunePanelRows = 0, kTuneJacobiWarps = 1, kTuneSplitkPerSM = 2 };
constexpr int kTuneKnobs = 3;
constexpr int kTuneClasses = 5;
int tune_class(int64_t size);
int tune_value(TuneKnob knob, int64_t size);

// The two timing events of an entry point, destroyed on every return path.
struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  EventPair() = default;
  EventPair(const EventPair&) = delete;
  EventPair& operator=(const EventPair&) = delete;
  ~EventPair() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// ---- gemm.cu ----
// C = alpha op(A) op(B) + beta C (+ diag_add on the diagonal), FP64 DMMA tiles.
// uplo == LOWER computes and writes only the lower triangle of C (SYRK use).
// `splitk_ws` (may be null) is scratch for split-K partial sums: at least
// gemm_splitk_ws_elems(m, n) doubles.  Without it no split-K is used.
qdwhp_status gemm(cudaStream_t st, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                  int64_t ldc, Uplo uplo = FULL, double diag_add = 0.0, double* splitk_ws = nullptr,
                  size_t splitk_ws_elems = 0);
size_t gemm_splitk_ws_elems(int64_t m, int64_t n);

// ---- ozaki.cu ----
// FP64 GEMM emulated on the BF16 tensor cores (Ozaki splitting: 9 balanced six-bit digits per entry,
// the 60 digit pairs with s + t <= 12, exact in FP32, FP64 accumulation).  Same operation as gemm(); needs
// gemm_ozaki_ws_bytes(m, n, k) bytes of scratch (16-byte aligned).
size_t gemm_ozaki_ws_bytes(int64_t m, int64_t n, int64_t k);
qdwhp_status gemm_ozaki(cudaStream_t st, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                        const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                        int64_t ldc, Uplo uplo, double diag_add, void* ws, size_t ws_bytes);
// Per host thread: while a scratch is installed, gemm() routes products with m, n >= 128 and
// k >= 256 whose scratch fits to gemm_ozaki (the emulated-precision solves install it).
struct EmulationScope {
  EmulationScope(void* ws, size_t bytes);
  ~EmulationScope();
  void* prev_ws;
  size_t prev_bytes;
};
// FP32 (reduced-precision QDWH steps): on the CUDA cores, or, with an Fp32TensorScope installed,
// products with m, n, k >= 256 as the BF16x6 split on the tensor cores (bf16x6.cu).
qdwhp_status gemm(cudaStream_t st, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha, const float* A,
                  int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc, Uplo uplo = FULL,
                  float diag_add = 0.0f);
// ---- bf16x6.cu ----
// FP32-accurate product from six BF16 slice products on tcgen05 (three slices per operand,
// FP32 accumulation); needs gemm_bf16x6_ws_bytes(m, n, k) bytes of scratch (16-byte aligned).
size_t gemm_bf16x6_ws_bytes(int64_t m, int64_t n, int64_t k);
qdwhp_status gemm_bf16x6(cudaStream_t st, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha,
                         const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                         Uplo uplo, float diag_add, void* ws, size_t ws_bytes);
// Per host thread: while a scratch is installed, the FP32 gemm() routes products with
// m, n, k >= 256 whose scratch fits to gemm_bf16x6.
struct Fp32TensorScope {
  Fp32TensorScope(void* ws, size_t bytes);
  ~Fp32TensorScope();
  void* prev_ws;
  size_t prev_bytes;
};

// ---- elementwise.cu ----
// Y = alpha X + beta Y (+ diag_add on the diagonal); beta == 0 never reads Y.
qdwhp_status axpby(cudaStream_t st, int64_t m, int64_t n, double alpha, const double* X, int64_t ldx,
                   double beta, double* Y, int64_t ldy, double diag_add = 0.0);
// Y = a Y + b Z, and (optional) partial sums of ||Y_new - Y_old||_F^2 into `diff_part`
// (kDiffParts doubles, summed by the caller's reduction).
constexpr int kDiffParts = 1024;
qdwhp_status axpby_diff(cudaStream_t st, int64_t m, int64_t n, double a, double* Y, int64_t ldy, double b,
                        const double* Z, int64_t ldz, double* diff_part);
qdwhp_status copy_matrix(cudaStream_t st, int64_t m, int64_t n, const double* X, int64_t ldx, double* Y,
                         int64_t ldy);
qdwhp_status set_matrix(cudaStream_t st, int64_t m, int64_t n, double offdiag, double diag, double* Y,
                        int64_t ldy);
// FP32 versions (reduced-precision QDWH steps) and precision conversion.
qdwhp_status axpby(cudaStream_t st, int64_t m, int64_t n, float alpha, const float* X, int64_t ldx, float beta,
                   float* Y, int64_t ldy, float diag_add = 0.0f);
qdwhp_status axpby_diff(cudaStream_t st, int64_t m, int64_t n, float a, float* Y, int64_t ldy, float b,
                        const float* Z, int64_t ldz, double* diff_part);
qdwhp_status copy_matrix(cudaStream_t st, int64_t m, int64_t n, const float* X, int64_t ldx, float* Y, int64_t ldy);
qdwhp_status set_matrix(cudaStream_t st, int64_t m, int64_t n, float offdiag, float diag, float* Y, int64_t ldy);
qdwhp_status convert(cudaStream_t st, int64_t m, int64_t n, const double* X, int64_t ldx, float* Y, int64_t ldy);
qdwhp_status convert(cudaStream_t st, int64_t m, int64_t n, const float* X, int64_t ldx, double* Y, int64_t ldy);
// R (n x n) = upper triangle of A, zeros below.
qdwhp_status copy_upper(cudaStream_t st, int64_t n, const double* A, int64_t lda, double* R, int64_t ldr);
// G (n x n) = R^T, R the upper triangle of the leading n x n block of A.
qdwhp_status copy_upper_t(cudaStream_t st, int64_t n, const double* A, int64_t lda, double* G, int64_t ldg);
// H := (H + H^T) / 2 (n x n).
qdwhp_status symmetrize_avg(cudaStream_t st, int64_t n, double* H, int64_t ldh);
// B (cols x rows, ld ldb) = A^T for A rows x cols (ld lda).
qdwhp_status transpose(cudaStream_t st, int64_t rows, int64_t cols, const double* A, int64_t lda, double* B,
                       int64_t ldb);
// Fills the lower triangle's mirror: Y(i, j) = Y(j, i) for i < j (n x n).
qdwhp_status symmetrize_from_lower(cudaStream_t st, int64_t n, double* Y, int64_t ldy);
// Sum of kDiffParts partials -> out (device scalar); also checks finiteness of the sum.
qdwhp_status reduce_parts(cudaStream_t st, const double* parts, int nparts, double* out);
// Count of non-finite entries of X (m x n) added into *count_dev (unsigned).
qdwhp_status count_nonfinite(cudaStream_t st, int64_t m, int64_t n, const double* X, int64_t ldx,
                             unsigned* count_dev);

// ---- chol.cu ----
constexpr int kCholNB = 64;
size_t potrf_linv_elems(int64_t n);
// Lower Cholesky in place; Linv receives the inverses of the kCholNB diagonal blocks;
// *fail_dev (int, device) receives the first failing 1-based column; the caller zeroes
// it beforehand and it is never cleared here, so it accumulates over calls.  Needs a
// scratch of potrf_scratch_elems(n) doubles.
size_t potrf_scratch_elems(int64_t n);
qdwhp_status potrf(cudaStream_t st, int64_t n, double* Z, int64_t ldz, double* Linv, double* scratch,
                   int* fail_dev);
// X (m x n) := X L^{-T} (trans) or X L^{-1} (!trans), L from potrf with its Linv blocks.
size_t trsm_scratch_elems(int64_t m, int64_t n);
qdwhp_status trsm_right_lower(cudaStream_t st, bool trans, int64_t m, int64_t n, double* X, int64_t ldx,
                              const double* L, int64_t ldl, const double* Linv, double* scratch);
// FP32 versions (reduced-precision QDWH steps).
qdwhp_status potrf(cudaStream_t st, int64_t n, float* Z, int64_t ldz, float* Linv, float* scratch, int* fail_dev);
qdwhp_status trsm_right_lower(cudaStream_t st, bool trans, int64_t m, int64_t n, float* X, int64_t ldx,
                              const float* L, int64_t ldl, const float* Linv, float* scratch);

// ---- qr.cu ----
constexpr int kQRNB = 32;
constexpr int kQROuter = 256;
struct QRFactors {
  double* Vall = nullptr;   // m x n explicit reflectors (unit diagonal, zeros above), ld = m
  double* T = nullptr;      // nblocks x kQRNB x kQRNB upper-triangular block factors
  double* To = nullptr;     // qr_to_elems(n): the same for the kQROuter-wide outer blocks
  double* tau = nullptr;    // n
  double* diagR = nullptr;  // n: R_ii
  int64_t m = 0, n = 0;
  int64_t band = 0;         // > 0: the matrix is [X; D] with X band x n and D diagonal (see geqrf)
};
size_t qr_scratch_elems(int64_t m, int64_t n);
size_t qr_to_elems(int64_t n);
// Householder QR of A (m x n, m >= n) in place: R in the upper triangle of A.  band > 0 declares
// A = [X; D] with X band x n and D n x n diagonal (band + n = m): the reflector of column j is
// then zero below row band + j, so every panel, trailing update and Q application works on the
// rows [j, band + j + width) only, which skips the zero part of the stacked matrix of a
// QR-based QDWH step (about 1/3 of its QR flops at m = 2n) without changing the arithmetic.
qdwhp_status geqrf(cudaStream_t st, int64_t m, int64_t n, double* A, int64_t lda, QRFactors& f,
                   double* scratch, int64_t band = 0);
// C (m x ncols) := Q [0; I; 0] restricted to columns col0 .. col0+ncols-1 of Q (explicit Q columns).
qdwhp_status orgqr_columns(cudaStream_t st, const QRFactors& f, int64_t col0, int64_t ncols, double* C,
                           int64_t ldc, double* scratch);
// C (m x ncols) := Q C with the full Q of the factorisation (scratch as for orgqr_columns).
qdwhp_status ormqr_left(cudaStream_t st, const QRFactors& f, double* C, int64_t ncols, int64_t ldc, double* scratch);

}  // namespace qdwhp
