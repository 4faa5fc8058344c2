// Full (thin) SVD by QDWH-SVD (Section 3.2).
//
// A (m x n, m >= n; m < n is solved on A^T with U and V swapped, Section 4.2) is scaled by
// alpha, the Lanczos estimate of ||A||_2 on A^T A, and QDWH computes its polar factor U_p
// (eqs. practical-polar-qr while c_k > 100, then practical-polar-chol) from ell_0 = 1e-15,
// which settles every singular value down to 1e-15 alpha.  H = U_p^T A is symmetric
// positive semidefinite with the singular values of A as eigenvalues; its
// eigendecomposition H = V Sigma V^T comes from the QDWH divide-and-conquer solver of dc.cu,
// and U = U_p V.  An eigenvalue of H that rounding made negative gives sigma = |lambda| and
// negates the column of U (A v = U_p H v = lambda U_p v).
//
// Null directions: QDWH maps singular values far below ell_0 alpha to values below 1, so
// U_p is not orthonormal there.  When the smallest computed sigma is at most kOrthFix alpha,
// U is replaced by the orthonormal factor of its Householder QR, signed by diag(R): columns
// that are already orthonormal change only by rounding, the others become an orthonormal
// completion (any completion is a valid set of singular vectors for sigma ~ 0).
#include <cmath>
#include <cstring>

#include "dc.h"

namespace qdwhp {

namespace {

constexpr double kGesvdEll0 = 1e-15;
constexpr double kOrthFix = 1e-14;
constexpr int kGesvdLanczosSteps = 30;
constexpr int kGesvdMaxSweeps = 30;
constexpr uint64_t kGesvdSeed = 0x51D5EEDull;

__global__ void abs_sign_kernel(int n, const double* lam, double* absval, double* sgn) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double v = lam[i];
    absval[i] = fabs(v);
    sgn[i] = v < 0.0 ? -1.0 : 1.0;
  }
}

// U(j, j) = sign(R_jj) (+1 for 0) on a zeroed U: then Q U is Q with its columns signed.
__global__ void signed_unit_diag_kernel(int n, const double* diagR, double* U, int64_t ldu) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    U[j + (int64_t)j * ldu] = diagR[j] < 0.0 ? -1.0 : 1.0;
}

struct GesvdWs {
  DcWs dc;                  // eigensolver of H (order n)
  QdwhWs q;                 // polar decomposition of the m x n A / alpha (QR-based steps)
  Schedule* sched = nullptr;
  LanczosState* lst = nullptr;
  double* lws = nullptr;
  unsigned* nonfinite = nullptr;
  double* X = nullptr;      // m x n: A / alpha, then U_p
  double* At = nullptr;     // A^T when the input is wide
  double* lam = nullptr;    // n eigenvalues of H (unordered)
  double* absval = nullptr; // n
  double* sgn = nullptr;    // n
  int* order = nullptr;     // n
  int* count = nullptr;
  double* Vraw = nullptr;   // n x n eigenvectors of H (unordered)
  char* emu = nullptr;
  size_t emu_bytes = 0;
};

void carve_gesvd(Arena& ar, int64_t m, int64_t n, bool need_transpose, bool emulated, GesvdWs& w) {
  carve_dc(ar, n, w.dc);
  carve_qdwh(ar, m, n, true, w.q, false);
  w.sched = ar.take<Schedule>(1);
  w.lst = ar.take<LanczosState>(1);
  w.lws = ar.take<double>(lanczos_ws_elems(m, n, kGesvdLanczosSteps));
  w.nonfinite = ar.take<unsigned>(4);
  w.X = ar.take<double>((size_t)m * n);
  if (need_transpose) w.At = ar.take<double>((size_t)m * n);
  w.lam = ar.take<double>(n);
  w.absval = ar.take<double>(n);
  w.sgn = ar.take<double>(n);
  w.order = ar.take<int>(n);
  w.count = ar.take<int>(4);
  w.Vraw = ar.take<double>((size_t)n * n);
  if (emulated) {
    w.emu_bytes = gemm_ozaki_ws_bytes(m, m, m);
    w.emu = ar.take<char>(w.emu_bytes);
  }
}

template <typename T>
qdwhp_status read_sync(cudaStream_t st, T* host, const T* dev, size_t count = 1) {
  QDWHP_CUDA_TRY(cudaMemcpyAsync(host, dev, sizeof(T) * count, cudaMemcpyDeviceToHost, st));
  QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  return QDWHP_OK;
}

// m >= n.  U: m x n (ldu), V: n x n (ldv).
qdwhp_status gesvd_impl(const double* A, int64_t m, int64_t n, int64_t lda, double* sigma, double* U, int64_t ldu,
                        double* V, int64_t ldv, GesvdWs& w, qdwhp_gesvd_info* inf, cudaStream_t st) {
  QDWHP_CUDA_TRY(cudaMemsetAsync(w.nonfinite, 0, sizeof(unsigned), st));
  QDWHP_TRY(count_nonfinite(st, m, n, A, lda, w.nonfinite));
  unsigned nonfinite = 0;
  QDWHP_TRY(read_sync(st, &nonfinite, w.nonfinite));
  if (nonfinite) return QDWHP_ERR_NONFINITE;
  // alpha >= ||A||_2 (to Lanczos accuracy): largest Ritz value of A^T A plus its residual
  QDWHP_TRY(lanczos(st, true, m, n, A, lda, kGesvdLanczosSteps, kGesvdSeed, w.lws, w.lst));
  LanczosState lst;
  QDWHP_TRY(read_sync(st, &lst, w.lst));
  if (lst.nonfinite) return QDWHP_ERR_NONFINITE;
  const double alpha = std::sqrt(std::max(lst.out[2] + lst.out[3], 0.0));
  if (!std::isfinite(alpha)) return QDWHP_ERR_NONFINITE;
  inf->alpha = alpha;
  if (!(alpha > 0.0)) {
    // the zero matrix: sigma = 0, any orthonormal U and V
    QDWHP_CUDA_TRY(cudaMemsetAsync(sigma, 0, sizeof(double) * n, st));
    QDWHP_TRY(set_matrix(st, m, n, 0.0, 1.0, U, ldu));
    return set_matrix(st, n, n, 0.0, 1.0, V, ldv);
  }

  // polar factor U_p of A / alpha
  QDWHP_TRY(dwh_schedule(st, nullptr, kGesvdEll0, 0, 100.0, w.sched));
  Schedule sched;
  QDWHP_TRY(read_sync(st, &sched, w.sched));
  QDWHP_TRY(axpby(st, m, n, 1.0 / alpha, A, lda, 0.0, w.X, m));
  QDWHP_CUDA_TRY(cudaMemsetAsync(w.q.fail, 0, sizeof(int), st));
  int n_qr = 0, n_chol = 0, n_f32 = 0;
  QDWHP_TRY(run_schedule(st, m, n, w.X, m, sched, false, w.q, &n_qr, &n_chol, &n_f32));
  inf->it_qr = n_qr;
  inf->it_chol = n_chol;
  int fail = 0;
  QDWHP_TRY(read_sync(st, &fail, w.q.fail));
  if (fail) return QDWHP_ERR_BREAKDOWN;

  // H = U_p^T A, symmetrised; H = V Lambda V^T
  QDWHP_TRY(gemm(st, true, false, n, n, m, 1.0, w.X, m, A, lda, 0.0, w.dc.M, n));
  QDWHP_TRY(symmetrize_avg(st, n, w.dc.M, n));
  DcStats stats;
  QDWHP_TRY(sym_eig_dc(st, n, -0.01 * alpha, 1.01 * alpha, kGesvdSeed, true, kGesvdMaxSweeps, w.lam, w.Vraw, n,
                       w.dc, &stats));
  inf->nodes = stats.nodes;
  inf->leaves = stats.leaves;
  inf->depth = stats.depth;
  inf->jacobi_sweeps = stats.jacobi_sweeps;
  inf->max_offblock = stats.max_offblock;
  inf->median_splits = stats.median_splits;

  // sigma = |lambda| descending; V unsigned, U = U_p (V sign(lambda))
  abs_sign_kernel<<<ceil_div(n, 256), 256, 0, st>>>((int)n, w.lam, w.absval, w.sgn);
  QDWHP_LAUNCH_CHECK();
  QDWHP_TRY(select_sort(st, n, w.absval, -1.0, INFINITY, w.order, w.count));
  QDWHP_TRY(gather_values(st, n, w.absval, w.order, sigma));
  QDWHP_TRY(gather_columns(st, n, n, w.Vraw, n, w.order, nullptr, V, ldv));
  QDWHP_TRY(gather_columns(st, n, n, w.Vraw, n, w.order, w.sgn, w.dc.W, n));
  QDWHP_TRY(gemm(st, false, false, m, n, n, 1.0, w.X, m, w.dc.W, n, 0.0, U, ldu));

  double smin = 0.0;
  QDWHP_TRY(read_sync(st, &smin, sigma + (n - 1)));
  if (!std::isfinite(smin)) return QDWHP_ERR_NONFINITE;
  if (smin <= kOrthFix * alpha) {
    inf->orthonormalized = 1;
    QDWHP_TRY(geqrf(st, m, n, U, ldu, w.q.qf, w.q.qr_scratch));
    QDWHP_TRY(set_matrix(st, m, n, 0.0, 0.0, U, ldu));
    signed_unit_diag_kernel<<<ceil_div(n, 256), 256, 0, st>>>((int)n, w.q.qf.diagR, U, ldu);
    QDWHP_LAUNCH_CHECK();
    QDWHP_TRY(ormqr_left(st, w.q.qf, U, n, ldu, w.q.qr_scratch));
  }
  return QDWHP_OK;
}

bool precision_ok(int32_t p) { return p == QDWHP_FP64 || p == QDWHP_FP64_EMULATED; }

}  // namespace

size_t gesvd_square_ws_bytes(int64_t n) {
  Arena ar;
  ar.dry = true;
  GesvdWs w;
  carve_gesvd(ar, n, n, false, false, w);
  return ar.used;
}

qdwhp_status gesvd_square(cudaStream_t st, int64_t n, const double* R, int64_t ldr, double* sigma, double* U,
                          int64_t ldu, double* V, int64_t ldv, void* ws, size_t ws_bytes, int* sweeps) {
  Arena ar{(char*)ws, ws_bytes};
  GesvdWs w;
  carve_gesvd(ar, n, n, false, false, w);
  if (!ar.ok()) return QDWHP_ERR_NOMEM;
  qdwhp_gesvd_info inf;
  memset(&inf, 0, sizeof(inf));
  QDWHP_TRY(gesvd_impl(R, n, n, ldr, sigma, U, ldu, V, ldv, w, &inf, st));
  if (sweeps) *sweeps = inf.jacobi_sweeps;
  return QDWHP_OK;
}

}  // namespace qdwhp

using namespace qdwhp;

extern "C" {

QDWHP_API size_t qdwhp_gesvd_workspace_bytes(int64_t m, int64_t n, int32_t precision) {
  if (m < 1 || n < 1 || !precision_ok(precision)) return 0;
  Arena ar;
  ar.dry = true;
  GesvdWs w;
  carve_gesvd(ar, std::max(m, n), std::min(m, n), m < n, precision == QDWHP_FP64_EMULATED, w);
  return ar.used;
}

QDWHP_API qdwhp_status qdwhp_gesvd_f64(const double* A, int64_t m, int64_t n, int64_t lda, int32_t precision,
                                       double* sigma, double* U, int64_t ldu, double* V, int64_t ldv,
                                       void* workspace, size_t ws_bytes, qdwhp_gesvd_info* info, void* stream) {
  if (!A || !sigma || !U || !V || m < 1 || n < 1 || lda < m || ldu < m || ldv < n) return QDWHP_ERR_ARG;
  if (!precision_ok(precision) || std::max(m, n) > (1 << 20) || std::min(m, n) > (1 << 17)) return QDWHP_ERR_ARG;
  if (!workspace || ws_bytes < qdwhp_gesvd_workspace_bytes(m, n, precision)) return QDWHP_ERR_NOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t mm = std::max(m, n), nn = std::min(m, n);
  Arena ar{(char*)workspace, ws_bytes};
  GesvdWs w;
  carve_gesvd(ar, mm, nn, m < n, precision == QDWHP_FP64_EMULATED, w);
  if (!ar.ok()) return QDWHP_ERR_NOMEM;
  EmulationScope emu_scope(w.emu, w.emu_bytes);
  qdwhp_gesvd_info inf;
  memset(&inf, 0, sizeof(inf));
  EventPair ev;
  QDWHP_CUDA_TRY(cudaEventCreate(&ev.e0));
  QDWHP_CUDA_TRY(cudaEventCreate(&ev.e1));
  QDWHP_CUDA_TRY(cudaEventRecord(ev.e0, st));
  qdwhp_status rc;
  if (m >= n) {
    rc = gesvd_impl(A, m, n, lda, sigma, U, ldu, V, ldv, w, &inf, st);
  } else {
    // A^T (n x m) = V Sigma U^T: the roles of U and V swap
    rc = transpose(st, m, n, A, lda, w.At, n);
    if (rc == QDWHP_OK) rc = gesvd_impl(w.At, n, m, n, sigma, V, ldv, U, ldu, w, &inf, st);
  }
  if (rc == QDWHP_OK) {
    float ms = 0.f;
    if (cudaEventRecord(ev.e1, st) == cudaSuccess && cudaEventSynchronize(ev.e1) == cudaSuccess)
      cudaEventElapsedTime(&ms, ev.e0, ev.e1);
    inf.ms_total = ms;
  }
  if (info) *info = inf;
  return rc;
}

}  // extern "C"
