// QDWHpartial-EIG (Algorithm 1) and QDWHpartial-SVD (Algorithm 2) drivers and the
// solver entry points of the C ABI.
//
// Every step runs in this library's kernels; the host enqueues them on the caller's
// stream and reads back a handful of scalars at stage boundaries (spectral bounds,
// the threshold, the subspace size ell, the count of captured pairs, Jacobi
// convergence) because they decide launch shapes and control flow.
//
// Readings where the paper is silent (also stated in the oracle):
//   * the wanted side is made negative by A' = eps A (eps = -1 for LARGEST) and the
//     threshold t' by a shift, B = A' - t' I (remark after Algorithm 1);
//   * mu = lam_lo - t', lam_lo = Lanczos lower bound (Ritz value - residual, pushed
//     1 % of the spread outwards); Algorithm 1 step 1 scales by |mu|;
//   * a requested count k becomes a threshold through the k-th Ritz value of a
//     (k+p)-dimensional subspace (Cauchy interlacing guarantees >= k pairs beyond it);
//   * the wanted width is kept >= guard * spread (default 10 %, unwanted side scaled by <= ~9);
//   * QR-based QDWH steps while c_k > c_qr (default 100), Section 4.2.
#include <cstdio>

#include "dc.h"
#include "internal.h"
#include "krylov.h"
#include "qdwh.h"

namespace qdwhp {

namespace {
thread_local char g_err[512] = "";
}

void set_last_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_err, sizeof(g_err), "%s (%s) at %s:%d: %s", cudaGetErrorName(e), what, file, line,
           cudaGetErrorString(e));
}

void set_error_message(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

namespace {

// lambda[i] = A(i, i), i < k: the Rayleigh quotients of the first k unit vectors.
__global__ void diag_copy_kernel(int k, const double* A, int64_t lda, double* lambda) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) lambda[i] = A[i + (int64_t)i * lda];
}

__global__ void index_scan_kernel(int n, const double* diagR, double tol, int* ind) {
  __shared__ int best;
  if (threadIdx.x == 0) best = n;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (fabs(diagR[i]) < tol) atomicMin(&best, i);
  __syncthreads();
  if (threadIdx.x == 0) *ind = best;
}

// Block Krylov bases of the count-to-threshold step wider than min(n / 8, this) keep only the
// last block: a wider basis would make its Rayleigh-Ritz problem cost as much as the solve.
constexpr int64_t kKrylovMaxCols = 2048;
// Such wide blocks take the stochastic Lanczos quadrature estimate instead from this order on
// (below it the block's Ritz-value bound captures fewer unwanted eigenvalues): kSlqProbes start
// vectors, kSlqSteps Lanczos steps each, kSlqZ standard errors of margin.
constexpr int64_t kSlqMinN = 1024;
// The SVD's reduced problem (the SVD of R from A Q2 = Q_C R) goes to one-sided Jacobi up to this
// order and to QDWH-SVD above it: a Jacobi sweep rotates every column about ell times, and the
// rounding of ~10 sweeps of those rotations left ~50 u per column in the singular values and
// vectors at ell ~ 1000 (a 3910 x 3733 SVD at k = 623: residual 1.2e-13 against the oracle's
// 5e-15), where QDWH-SVD's Rayleigh-quotient eigenvalues of H stay at the rounding level.
constexpr int64_t kSvdJacobiMax = 512;
constexpr int kSlqProbes = 16;
constexpr int kSlqSteps = 64;
constexpr double kSlqZ = 3.0;
constexpr uint64_t kStreamSlq = 0x534C5150ull;   // "SLQP"
constexpr int kLanczosMaxSteps = 64;
uint64_t slq_probe_seed(uint64_t seed, int j) { return seed ^ kStreamSlq ^ ((uint64_t)(j + 1) * 0x9E3779B97F4A7C15ull); }
// Stopping tolerance of the reduced-problem Jacobi when its vectors are used: the
// normalised off-diagonal inner products (computed in double-double) down to ~2u.
constexpr double kJacobiTight = 4.5e-16;

// Precision modes: Cholesky-based steps but the last in FP32, and/or the FP64 products
// emulated on the BF16 tensor cores.
bool fp32_steps(const qdwhp_opts& o) { return o.precision == QDWHP_MIXED || o.precision == QDWHP_MIXED_EMULATED; }
bool emulated_products(const qdwhp_opts& o) {
  return o.precision == QDWHP_FP64_EMULATED || o.precision == QDWHP_MIXED_EMULATED;
}

struct Common {
  // small-problem and control buffers shared by both drivers
  LanczosState* lst = nullptr;
  LanczosState* slq = nullptr;   // EIG: the probes of the stochastic count-to-threshold estimate
  JacobiState* jst = nullptr;
  Schedule* sched = nullptr;
  ZoloSchedule* zsched = nullptr;
  int* ints = nullptr;        // [0] ind, [1] count, [2..] spare
  unsigned* nonfinite = nullptr;
  double* vals = nullptr;     // n
  int* order = nullptr;       // n
  double* lws = nullptr;      // Lanczos workspace
  double* splitk = nullptr;
  size_t splitk_elems = 0;
};

// Pinned host staging for scalars read back from the device.
struct HostScalars {
  LanczosState lst;
  JacobiState jst;
  Schedule sched;
  ZoloSchedule zsched;
  int ints[4];
  unsigned nonfinite;
};

void carve_common(Arena& ar, int64_t m, int64_t n, int steps, Common& c) {
  c.lst = ar.take<LanczosState>(1);
  c.slq = ar.take<LanczosState>(kSlqProbes);
  c.jst = ar.take<JacobiState>(1);
  c.sched = ar.take<Schedule>(1);
  c.zsched = ar.take<ZoloSchedule>(1);
  c.ints = ar.take<int>(8);
  c.nonfinite = ar.take<unsigned>(4);
  c.vals = ar.take<double>(std::max<int64_t>(n, 1));
  c.order = ar.take<int>(std::max<int64_t>(n, 1));
  (void)steps;
  c.lws = ar.take<double>(lanczos_ws_elems(m, n, kLanczosMaxSteps));
  c.splitk_elems = std::min<size_t>(gemm_splitk_ws_elems(std::min<int64_t>(n, 2048), std::min<int64_t>(n, 2048)),
                                    size_t(8) << 20);
  c.splitk = ar.take<double>(c.splitk_elems);
}

int64_t resolve_k(int64_t n, const qdwhp_opts& o, int64_t k_arg) {
  if (k_arg > 0) return k_arg;
  if (o.count > 0) return o.count;
  return qdwhp_k_from_fraction(n, o.fraction);
}

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) cudaEventRecord(e0, st);
  }
  float stop() {
    float ms = 0.f;
    if (e0 && e1) {
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    return ms;
  }
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

qdwhp_status sync_read(cudaStream_t st, void* host, const void* dev, size_t bytes) {
  QDWHP_CUDA_TRY(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st));
  QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  return QDWHP_OK;
}

// Orthonormal basis of the columns of Y (rows x b): Householder QR then explicit Q.
qdwhp_status orth(cudaStream_t st, int64_t rows, int64_t b, double* Y, double* Qout, QRFactors& f, double* scratch) {
  QDWHP_TRY(geqrf(st, rows, b, Y, rows, f, scratch));
  return orgqr_columns(st, f, 0, b, Qout, rows, scratch);
}

// ---------------------------------------------------------------------------------------
struct EigWs {
  Common c;
  QdwhWs q;
  QRFactors f;
  double* qr_scratch = nullptr;
  double* X = nullptr;   // n x n iterate
  double* S1 = nullptr;  // n x n capacity: M (Rayleigh-Ritz matrix) / H
  double* S2 = nullptr;  // n x n capacity: G, then M V, then gathered W
  double* S3 = nullptr;  // n x n capacity: Vj
  bool has_dc = false;   // n > kDcMin: Rayleigh-Ritz problems may need divide and conquer
  DcWs dc;               // its own buffers; the large ones are lent from the above at run time
  int dc_nodes = 0;      // splits of the last divide-and-conquer solve
  char* emu = nullptr;   // emulated FP64 products: their scratch
  size_t emu_bytes = 0;
  char* f32tc = nullptr; // FP32 products of the reduced-precision steps on the tensor cores: their scratch
  size_t f32tc_bytes = 0;
};

void carve_eig(Arena& ar, int64_t n, const qdwhp_opts& o, EigWs& w) {
  carve_common(ar, n, n, o.lanczos_steps, w.c);
  carve_qdwh(ar, n, n, o.zolo_r > 0, w.q, fp32_steps(o), o.zolo_r > 0);
  w.X = ar.take<double>((size_t)n * n);
  w.f.Vall = ar.take<double>((size_t)n * n);
  w.f.T = ar.take<double>((size_t)ceil_div(n, kQRNB) * kQRNB * kQRNB);
  w.f.To = ar.take<double>(qr_to_elems(n));
  w.f.tau = ar.take<double>(n);
  w.f.diagR = ar.take<double>(n);
  w.qr_scratch = ar.take<double>(qr_scratch_elems(n, n));
  w.S1 = ar.take<double>((size_t)n * n);
  w.S2 = ar.take<double>((size_t)n * n);
  w.S3 = ar.take<double>((size_t)n * n);
  w.has_dc = n > kDcMin;
  if (w.has_dc) carve_dc_own(ar, n, w.dc);
  if (emulated_products(o)) {
    w.emu_bytes = gemm_ozaki_ws_bytes(n, n, n);
    w.emu = ar.take<char>(w.emu_bytes);
  }
  if (fp32_steps(o)) {
    w.f32tc_bytes = gemm_bf16x6_ws_bytes(n, n, n);
    w.f32tc = ar.take<char>(w.f32tc_bytes);
  }
}

// Eigenvalues (into w.c.vals) and eigenvectors (S3, ld ell) of the symmetric ell x ell
// matrix in S1, whose spectrum lies in [lower, upper].  Up to kDcMin: one-sided Jacobi with
// Rayleigh quotients; larger: QDWH spectral divide and conquer (S1 is then destroyed), run in
// the buffers that are dead at this point (X, S2, the extraction QR, q.Z).
// `values_only`: only the eigenvalues are used, and those are accurate to the square of
// the Jacobi off-diagonal tolerance, so a loose tolerance (1e-9) is enough.
qdwhp_status small_sym_eig(cudaStream_t st, int64_t ell, double lower, double upper, uint64_t seed, EigWs& w,
                           int max_sweeps, HostScalars& hs, int* sweeps, bool values_only = false) {
  w.dc_nodes = 0;
  QDWHP_TRY(symmetrize_avg(st, ell, w.S1, ell));
  if (ell > kDcMin && w.has_dc) {
    DcWs dv = w.dc;
    dv.M = w.S1;
    dv.X = w.X;
    dv.Q = w.S2;
    dv.W = w.q.Z;
    dv.f = w.f;
    dv.qr_scratch = w.qr_scratch;
    DcStats stats;
    QDWHP_TRY(sym_eig_dc(st, ell, lower, upper, seed, !values_only, max_sweeps, w.c.vals, w.S3, ell, dv, &stats));
    *sweeps = stats.jacobi_sweeps;
    w.dc_nodes = stats.nodes;
    return QDWHP_OK;
  }
  // G = M - lower I is positive semidefinite; its right singular vectors are M's eigenvectors.
  QDWHP_TRY(axpby(st, ell, ell, 1.0, w.S1, ell, 0.0, w.S2, ell, -lower));
  int conv = 0;
  const double tol = values_only ? 1e-9 : kJacobiTight;
  QDWHP_TRY(jacobi_onesided(st, ell, ell, w.S2, ell, w.S3, ell, max_sweeps, tol, w.c.jst, &hs.jst, sweeps, &conv));
  if (!conv) return QDWHP_ERR_NOT_CONVERGED;
  // The accumulated rotations drift the column norms by O(rotations * u): rescale.
  QDWHP_TRY(normalize_columns(st, ell, ell, w.S3, ell, nullptr));
  // Rayleigh quotients v_i^T M v_i
  QDWHP_TRY(gemm(st, false, false, ell, ell, ell, 1.0, w.S1, ell, w.S3, ell, 0.0, w.S2, ell));
  return column_dots(st, ell, ell, w.S3, ell, w.S2, ell, w.c.vals);
}

qdwhp_status eig_impl(const double* A, int64_t n, int64_t lda, const qdwhp_opts& o, double* lambda, double* V,
                      int64_t ldv, void* workspace, size_t ws_bytes, qdwhp_info* info, cudaStream_t st) {
  const int64_t k = resolve_k(n, o, 0);
  if (k < 1 || k > n) return QDWHP_ERR_ARG;
  Arena ar{(char*)workspace, ws_bytes};
  EigWs w;
  carve_eig(ar, n, o, w);
  if (!ar.ok()) return QDWHP_ERR_NOMEM;
  EmulationScope emu_scope(w.emu, w.emu_bytes);
  Fp32TensorScope f32_scope(w.f32tc, w.f32tc_bytes);
  Timer timer(st);
  HostScalars hs;
  qdwhp_info inf;
  memset(&inf, 0, sizeof(inf));
  const double eps_side = (o.side == QDWHP_SMALLEST) ? 1.0 : -1.0;

  QDWHP_CUDA_TRY(cudaMemsetAsync(w.c.nonfinite, 0, sizeof(unsigned), st));
  QDWHP_TRY(count_nonfinite(st, n, n, A, lda, w.c.nonfinite));
  // Step 1: Lanczos bounds.
  QDWHP_TRY(lanczos(st, false, n, n, A, lda, o.lanczos_steps, o.seed, w.c.lws, w.c.lst));
  QDWHP_CUDA_TRY(cudaMemcpyAsync(&hs.nonfinite, w.c.nonfinite, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  QDWHP_TRY(sync_read(st, &hs.lst, w.c.lst, sizeof(LanczosState)));
  if (hs.nonfinite || hs.lst.nonfinite) return QDWHP_ERR_NONFINITE;
  const double th_min = hs.lst.out[0], r_min = hs.lst.out[1], th_max = hs.lst.out[2], r_max = hs.lst.out[3];
  double lo_raw, hi_raw;
  if (eps_side < 0) {
    lo_raw = -(th_max + r_max);
    hi_raw = -(th_min - r_min);
  } else {
    lo_raw = th_min - r_min;
    hi_raw = th_max + r_max;
  }
  // Degenerate case: the spectrum is one point to rounding (n = 1, a multiple of the identity,
  // the zero matrix).  mu would be 0 (Algorithm 1 scales by 1/|mu|) and every vector is an
  // eigenvector: the first k unit vectors and their Rayleigh quotients.
  if (hi_raw - lo_raw <= 16 * 1.1102230246251565e-16 * std::max(std::fabs(lo_raw), std::fabs(hi_raw))) {
    QDWHP_TRY(set_matrix(st, n, k, 0.0, 1.0, V, ldv));
    diag_copy_kernel<<<ceil_div(k, 256), 256, 0, st>>>((int)k, A, lda, lambda);
    QDWHP_LAUNCH_CHECK();
    inf.ms_total = timer.stop();
    inf.k = k;
    if (info) *info = inf;
    return QDWHP_OK;
  }
  const double spread = hi_raw - lo_raw;
  const double lam_lo = lo_raw - 0.01 * spread, lam_hi = hi_raw + 0.01 * spread;

  // Threshold for the requested count: block Krylov space of P = lam_hi I - A' from k + p
  // SplitMix64 vectors (each block orthonormalised before the next product), Rayleigh-Ritz of A'
  // on it, whose k-th Ritz value bounds the k-th eigenvalue (Cauchy interlacing).  When
  // (q+1) b > min(n/8, 2048) columns: for n >= kSlqMinN the stochastic Lanczos quadrature
  // estimate (an estimate only: the count check after Rayleigh-Ritz and the retries keep the
  // k pairs guaranteed), else, or if it finds no node, only the last block, P^(q+1) Om, is kept.
  const int64_t b = std::min<int64_t>(n, k + o.block_extra);
  const int q = o.power_steps > 0 ? o.power_steps : 6;
  const bool krylov = (int64_t)(q + 1) * b <= std::min<int64_t>(n / 8, kKrylovMaxCols);
  double theta_k = 0.0;
  bool have_theta = false;
  int sweeps = 0;
  if (!krylov && n >= kSlqMinN) {
    for (int j = 0; j < kSlqProbes; ++j)
      QDWHP_TRY(lanczos(st, false, n, n, A, lda, kSlqSteps, slq_probe_seed(o.seed, j), w.c.lws, w.c.slq + j));
    QDWHP_TRY(slq_threshold(st, w.c.slq, kSlqProbes, eps_side, n, k, kSlqZ, w.S1));
    double got[2];
    QDWHP_TRY(sync_read(st, got, w.S1, sizeof(got)));
    if (got[1] > 0.0 && std::isfinite(got[0])) {
      theta_k = got[0];
      have_theta = true;
    }
  }
  if (!have_theta) {
    const int64_t width = krylov ? (q + 1) * b : b;
    double* Y = w.X;           // n x b
    double* Kb = w.S3;         // n x width
    double* Qj = w.q.Z;        // n x b
    double* AK = w.q.Y;        // n x width
    QDWHP_TRY(fill_uniform(st, n, b, o.seed ^ kStreamBlock, Y, n));
    for (int j = 0; j <= q; ++j) {
      double* Qdst = krylov ? Kb + (int64_t)j * b * n : Qj;
      QDWHP_TRY(orth(st, n, b, Y, Qdst, w.f, w.qr_scratch));
      if (j < q || !krylov) {
        QDWHP_TRY(axpby(st, n, b, lam_hi, Qdst, n, 0.0, Y, n));
        QDWHP_TRY(gemm(st, false, false, n, b, n, -eps_side, A, lda, Qdst, n, 1.0, Y, n));
      }
    }
    if (krylov) {
      QDWHP_TRY(copy_matrix(st, n, width, Kb, n, AK, n));
      QDWHP_TRY(orth(st, n, width, AK, Kb, w.f, w.qr_scratch));
    } else {
      QDWHP_TRY(orth(st, n, b, Y, Kb, w.f, w.qr_scratch));
    }
    QDWHP_TRY(gemm(st, false, false, n, width, n, eps_side, A, lda, Kb, n, 0.0, AK, n));
    QDWHP_TRY(gemm(st, true, false, width, width, n, 1.0, Kb, n, AK, n, 0.0, w.S1, width, FULL, 0.0, w.c.splitk,
                   w.c.splitk_elems));
    QDWHP_TRY(small_sym_eig(st, width, lam_lo, lam_hi, o.seed, w, o.jacobi_max_sweeps, hs, &sweeps, true));
    QDWHP_TRY(select_sort(st, width, w.c.vals, 1.0, INFINITY, w.c.order, w.c.ints + 1));
    QDWHP_TRY(gather_values(st, 1, w.c.vals, w.c.order + (k - 1), w.S1));
  }
  // Step 2's polar iterations: QDWH (iters_eig Cholesky-based steps from ell_0 = s) or
  // Zolo-PD of order zolo_r until ell_k = 1.
  const bool zolo = o.zolo_r > 0;
  if (zolo) {
    QDWHP_TRY(zolo_schedule(st, o.s_eig, o.zolo_r, o.zolo_c_qr, w.c.zsched));
    QDWHP_CUDA_TRY(cudaMemcpyAsync(&hs.zsched, w.c.zsched, sizeof(ZoloSchedule), cudaMemcpyDeviceToHost, st));
  } else {
    // Cholesky-based in every iteration (Section 4.1; c_qr is the SVD's switch)
    QDWHP_TRY(dwh_schedule(st, nullptr, o.s_eig, o.iters_eig, INFINITY, w.c.sched));
    QDWHP_CUDA_TRY(cudaMemcpyAsync(&hs.sched, w.c.sched, sizeof(Schedule), cudaMemcpyDeviceToHost, st));
  }
  if (!have_theta) QDWHP_TRY(sync_read(st, &theta_k, w.S1, sizeof(double)));
  double t = theta_k + 1e-10 * spread;
  t = std::max(t, lam_lo + o.guard * (lam_hi - lam_lo));
  const double s = o.s_eig;

  int retries = 0;
  int64_t ell = 0;
  double mu = 0.0;
  int count = 0;
  for (;;) {
    mu = lam_lo - t;
    const double absmu = std::fabs(mu);
    // Steps 1-2: X0 = (1-s) B / |mu| - s I with B = eps A - t I.
    QDWHP_TRY(axpby(st, n, n, (1.0 - s) * eps_side / absmu, A, lda, 0.0, w.X, n, -((1.0 - s) * t / absmu + s)));
    QDWHP_CUDA_TRY(cudaMemsetAsync(w.q.fail, 0, sizeof(int), st));
    int n_qr = 0, n_chol = 0, n_f32 = 0;
    if (zolo) {
      QDWHP_TRY(run_zolo(st, n, n, w.X, n, hs.zsched, w.q, &n_qr, &n_chol));
    } else {
      QDWHP_TRY(run_schedule(st, n, n, w.X, n, hs.sched, fp32_steps(o), w.q, &n_qr, &n_chol, &n_f32));
    }
    inf.it_f32 = n_f32;
    inf.it_qr = n_qr;
    inf.it_chol = n_chol;
    // Step 3: QR of (r(A~) + I) / 2, or of (r(A~) + I) Omega / 2 with the Gaussian Omega of
    // Section 4.1 (S1 and S2 are free until Rayleigh-Ritz).
    QDWHP_TRY(axpby(st, n, n, 0.5, w.X, n, 0.0, w.X, n, 0.5));
    double* F = w.X;
    if (o.use_omega) {
      QDWHP_TRY(fill_gaussian(st, n, n, o.seed ^ kStreamOmega, 1.0 / std::sqrt((double)n), w.S2, n));
      QDWHP_TRY(gemm(st, false, false, n, n, n, 1.0, w.X, n, w.S2, n, 0.0, w.S1, n));
      F = w.S1;
    }
    QDWHP_TRY(geqrf(st, n, n, F, n, w.f, w.qr_scratch));
    // Step 4: index rule.
    index_scan_kernel<<<1, 1024, 0, st>>>((int)n, w.f.diagR, o.tol, w.c.ints);
    QDWHP_LAUNCH_CHECK();
    int fail = 0;
    double diffs[kMaxSteps];
    QDWHP_CUDA_TRY(cudaMemcpyAsync(&fail, w.q.fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    QDWHP_CUDA_TRY(cudaMemcpyAsync(diffs, w.q.diff, sizeof(double) * kMaxSteps, cudaMemcpyDeviceToHost, st));
    QDWHP_TRY(sync_read(st, hs.ints, w.c.ints, sizeof(int) * 4));
    if (fail) return QDWHP_ERR_BREAKDOWN;
    const int nsteps = zolo ? hs.zsched.nsteps : hs.sched.nsteps;
    for (int i = 0; i < nsteps && i < 12; ++i) {
      inf.conv[i] = std::sqrt(diffs[i]);
      inf.ell_k[i] = zolo ? hs.zsched.ell_after[i] : hs.sched.ell_after[i];
    }
    inf.zolo_steps = zolo ? nsteps : 0;
    const int ind = hs.ints[0];
    ell = n - ind;
    count = 0;
    if (ell > 0) {
      // Step 5: Q2 = trailing ell columns of Q.
      double* Q2 = w.q.Y;
      QDWHP_TRY(orgqr_columns(st, w.f, ind, ell, Q2, n, w.qr_scratch));
      // Step 6: Rayleigh-Ritz on the original A.
      double* AQ2 = w.q.Z;
      QDWHP_TRY(gemm(st, false, false, n, ell, n, 1.0, A, lda, Q2, n, 0.0, AQ2, n));
      QDWHP_TRY(gemm(st, true, false, ell, ell, n, 1.0, Q2, n, AQ2, n, 0.0, w.S1, ell, FULL, 0.0, w.c.splitk,
                     w.c.splitk_elems));
      const double a_lo = th_min - r_min - 0.01 * spread;   // bounds of A's spectrum
      const double a_hi = th_max + r_max + 0.01 * spread;
      QDWHP_TRY(small_sym_eig(st, ell, a_lo, a_hi, o.seed, w, o.jacobi_max_sweeps, hs, &sweeps));
      inf.jacobi_sweeps = sweeps;
      // wanted: eps * theta <= t, ordered ascending in eps * theta
      QDWHP_TRY(select_sort(st, ell, w.c.vals, eps_side, t, w.c.order, w.c.ints + 1));
      QDWHP_TRY(sync_read(st, hs.ints, w.c.ints, sizeof(int) * 4));
      count = hs.ints[1];
    }
    if (count >= k || retries >= o.max_retries) break;
    ++retries;
    t = t + 0.25 * (lam_hi - t);
  }
  if (count < k) return QDWHP_ERR_COUNT;
  // Step 7: the k wanted pairs, V = Q2 W.
  QDWHP_TRY(gather_values(st, k, w.c.vals, w.c.order, lambda));
  QDWHP_TRY(gather_columns(st, ell, k, w.S3, ell, w.c.order, nullptr, w.S2, ell));
  QDWHP_TRY(gemm(st, false, false, n, k, ell, 1.0, w.q.Y, n, w.S2, ell, 0.0, V, ldv));
  inf.ms_total = timer.stop();
  inf.retries = retries;
  inf.ell = ell;
  inf.k = k;
  inf.t = eps_side * t;
  inf.mu = eps_side * mu;
  inf.dc_nodes = w.dc_nodes;
  if (info) *info = inf;
  return QDWHP_OK;
}

// ---------------------------------------------------------------------------------------
struct SvdWs {
  Common c;
  QdwhWs q;
  QRFactors f;
  double* qr_scratch = nullptr;
  double* X = nullptr;    // m x n iterate
  double* C = nullptr;    // m x n capacity: A Q2 (and A Qb)
  double* Vj = nullptr;   // n x n capacity
  double* W = nullptr;    // n x n capacity: gathered V~
  double* At = nullptr;   // transposed input when m < n
  char* emu = nullptr;    // emulated FP64 products: their scratch
  size_t emu_bytes = 0;
  char* f32tc = nullptr;  // FP32 products of the reduced-precision steps on the tensor cores
  size_t f32tc_bytes = 0;
  char* rr = nullptr;     // QDWH-SVD of a reduced problem of order > kSvdJacobiMax: its scratch
  size_t rr_bytes = 0;
};

void carve_svd(Arena& ar, int64_t m, int64_t n, const qdwhp_opts& o, SvdWs& w, bool need_transpose) {
  carve_common(ar, m, n, o.lanczos_steps, w.c);
  carve_qdwh(ar, m, n, true, w.q, fp32_steps(o), o.zolo_r > 0);
  w.X = ar.take<double>((size_t)m * n);
  w.f.Vall = ar.take<double>((size_t)n * n);
  w.f.T = ar.take<double>((size_t)ceil_div(n, kQRNB) * kQRNB * kQRNB);
  w.f.To = ar.take<double>(qr_to_elems(n));
  w.f.tau = ar.take<double>(n);
  w.f.diagR = ar.take<double>(n);
  w.qr_scratch = ar.take<double>(qr_scratch_elems(n, n));
  w.C = ar.take<double>((size_t)m * n);
  w.Vj = ar.take<double>((size_t)n * n);
  w.W = ar.take<double>((size_t)n * n);
  if (need_transpose) w.At = ar.take<double>((size_t)m * n);
  if (emulated_products(o)) {
    const int64_t d = std::max(m, n);
    w.emu_bytes = gemm_ozaki_ws_bytes(d, d, d);
    w.emu = ar.take<char>(w.emu_bytes);
  }
  if (fp32_steps(o)) {
    const int64_t d = std::max(m, n);
    w.f32tc_bytes = gemm_bf16x6_ws_bytes(d, d, d);
    w.f32tc = ar.take<char>(w.f32tc_bytes);
  }
  if (n > kSvdJacobiMax) {
    w.rr_bytes = gesvd_square_ws_bytes(n);
    w.rr = ar.take<char>(w.rr_bytes);
  }
}

qdwhp_status svd_impl(const double* A, int64_t m, int64_t n, int64_t lda, int64_t k, const qdwhp_opts& o,
                      double* sigma, double* U, int64_t ldu, double* V, int64_t ldv, SvdWs& w, qdwhp_info* info,
                      cudaStream_t st) {
  Timer timer(st);
  HostScalars hs;
  qdwhp_info inf;
  memset(&inf, 0, sizeof(inf));
  QDWHP_CUDA_TRY(cudaMemsetAsync(w.c.nonfinite, 0, sizeof(unsigned), st));
  QDWHP_TRY(count_nonfinite(st, m, n, A, lda, w.c.nonfinite));
  // Step 1: alpha ~ ||A||_2 from Lanczos on A^T A.
  QDWHP_TRY(lanczos(st, true, m, n, A, lda, o.lanczos_steps, o.seed, w.c.lws, w.c.lst));
  QDWHP_CUDA_TRY(cudaMemcpyAsync(&hs.nonfinite, w.c.nonfinite, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  QDWHP_TRY(sync_read(st, &hs.lst, w.c.lst, sizeof(LanczosState)));
  if (hs.nonfinite || hs.lst.nonfinite) return QDWHP_ERR_NONFINITE;
  const double alpha = std::sqrt(std::max(hs.lst.out[2] + hs.lst.out[3], 0.0));
  if (!std::isfinite(alpha)) return QDWHP_ERR_NONFINITE;
  if (!(alpha > 0.0)) {
    // the zero matrix: every singular value is 0 and any orthonormal U, V serve
    QDWHP_CUDA_TRY(cudaMemsetAsync(sigma, 0, sizeof(double) * k, st));
    QDWHP_TRY(set_matrix(st, m, k, 0.0, 1.0, U, ldu));
    QDWHP_TRY(set_matrix(st, n, k, 0.0, 1.0, V, ldv));
    inf.ms_total = timer.stop();
    inf.k = k;
    if (info) *info = inf;
    return QDWHP_OK;
  }

  // Relative threshold s from the k-th Ritz value of A^T A on span((A^T A)^(q+1) Om), Om of
  // k + p SplitMix64 columns (subspace iteration, each block orthonormalised before the next
  // product).
  const int64_t b = std::min<int64_t>(n, k + o.block_extra);
  const int q = o.power_steps > 0 ? o.power_steps : 2;
  const int64_t width = b;
  double* Y = w.q.Y;     // n x b
  double* Kb = w.Vj;     // n x b
  double* T1 = w.X;      // m x b
  QDWHP_TRY(fill_uniform(st, n, b, o.seed ^ kStreamBlock, Y, n));
  for (int j = 0; j <= q; ++j) {
    QDWHP_TRY(orth(st, n, b, Y, Kb, w.f, w.qr_scratch));
    QDWHP_TRY(gemm(st, false, false, m, b, n, 1.0, A, lda, Kb, n, 0.0, T1, m));
    QDWHP_TRY(gemm(st, true, false, n, b, m, 1.0, A, lda, T1, m, 0.0, Y, n));
  }
  QDWHP_TRY(orth(st, n, b, Y, Kb, w.f, w.qr_scratch));
  QDWHP_TRY(gemm(st, false, false, m, width, n, 1.0, A, lda, Kb, n, 0.0, w.C, m));
  // Ritz values of A^T A on span(K) are the squared singular values of C = A K = Q_C R, i.e. of
  // R^T.  Forming C^T C instead would square the grading of the columns (they span decades of
  // sigma^2), which slows one-sided Jacobi; on R^T it needs about ten sweeps.
  QDWHP_TRY(geqrf(st, m, width, w.C, m, w.q.qf, w.q.qr_scratch));
  double* G = w.W;
  QDWHP_TRY(copy_upper_t(st, width, w.C, m, G, width));
  int sweeps = 0, conv = 0;
  // values only: singular value errors are of the order of the squared off-diagonal tolerance
  const double tol_b = 1e-9;
  QDWHP_TRY(jacobi_onesided(st, width, width, G, width, w.Vj, width, o.jacobi_max_sweeps, tol_b, w.c.jst, &hs.jst,
                            &sweeps, &conv));
  if (!conv) return QDWHP_ERR_NOT_CONVERGED;
  QDWHP_TRY(column_norms(st, width, width, G, width, w.c.vals));
  QDWHP_TRY(select_sort(st, width, w.c.vals, -1.0, INFINITY, w.c.order, w.c.ints + 1));
  QDWHP_TRY(gather_values(st, 1, w.c.vals, w.c.order + (k - 1), w.q.Z));
  double sig_hat = 0.0;
  QDWHP_TRY(sync_read(st, &sig_hat, w.q.Z, sizeof(double)));
  double s = std::max(sig_hat / alpha * (1.0 - 1e-10), 1e-15);

  int retries = 0;
  int64_t ell = 0;
  int count = 0;
  bool rr_unit = false;   // the reduced SVD came from QDWH-SVD (unit U columns) rather than Jacobi
  for (;;) {
    const bool zolo = o.zolo_r > 0;
    if (zolo) {
      QDWHP_TRY(zolo_schedule(st, s, o.zolo_r, o.zolo_c_qr, w.c.zsched));
      QDWHP_TRY(sync_read(st, &hs.zsched, w.c.zsched, sizeof(ZoloSchedule)));
    } else {
      QDWHP_TRY(dwh_schedule(st, nullptr, s, 0, o.c_qr, w.c.sched));
      QDWHP_TRY(sync_read(st, &hs.sched, w.c.sched, sizeof(Schedule)));
    }
    // Step 2: QDWH (or Zolo-PD) on A / alpha from ell_0 = s.
    QDWHP_TRY(axpby(st, m, n, 1.0 / alpha, A, lda, 0.0, w.X, m));
    QDWHP_CUDA_TRY(cudaMemsetAsync(w.q.fail, 0, sizeof(int), st));
    int n_f32 = 0;
    if (zolo) {
      QDWHP_TRY(run_zolo(st, m, n, w.X, m, hs.zsched, w.q, &inf.it_qr, &inf.it_chol));
    } else {
      QDWHP_TRY(run_schedule(st, m, n, w.X, m, hs.sched, fp32_steps(o), w.q, &inf.it_qr, &inf.it_chol,
                             &n_f32));
    }
    inf.it_f32 = n_f32;
    // Step 3: QR of I - X^T X.
    double* B = w.q.Z;
    QDWHP_TRY(gemm(st, true, false, n, n, m, -1.0, w.X, m, w.X, m, 0.0, B, n, LOWER, 1.0));
    QDWHP_TRY(symmetrize_from_lower(st, n, B, n));
    // or the QR of (I - X^T X) Omega (Section 4.1; W and Vj are free until the projection)
    double* F = B;
    if (o.use_omega) {
      QDWHP_TRY(fill_gaussian(st, n, n, o.seed ^ kStreamOmega, 1.0 / std::sqrt((double)n), w.W, n));
      QDWHP_TRY(gemm(st, false, false, n, n, n, 1.0, B, n, w.W, n, 0.0, w.Vj, n));
      F = w.Vj;
    }
    QDWHP_TRY(geqrf(st, n, n, F, n, w.f, w.qr_scratch));
    index_scan_kernel<<<1, 1024, 0, st>>>((int)n, w.f.diagR, o.tol, w.c.ints);
    QDWHP_LAUNCH_CHECK();
    int fail = 0;
    double diffs[kMaxSteps];
    QDWHP_CUDA_TRY(cudaMemcpyAsync(&fail, w.q.fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    QDWHP_CUDA_TRY(cudaMemcpyAsync(diffs, w.q.diff, sizeof(double) * kMaxSteps, cudaMemcpyDeviceToHost, st));
    QDWHP_TRY(sync_read(st, hs.ints, w.c.ints, sizeof(int) * 4));
    if (fail) return QDWHP_ERR_BREAKDOWN;
    const int nsteps = zolo ? hs.zsched.nsteps : hs.sched.nsteps;
    for (int i = 0; i < nsteps && i < 12; ++i) {
      inf.conv[i] = std::sqrt(diffs[i]);
      inf.ell_k[i] = zolo ? hs.zsched.ell_after[i] : hs.sched.ell_after[i];
    }
    inf.zolo_steps = zolo ? nsteps : 0;
    const int ind = hs.ints[0];
    ell = n - ind;
    count = 0;
    if (ell > 0) {
      // Steps 5-6: Q2, A Q2 and its SVD.  A Q2 = Q_C R (Householder), then one-sided Jacobi
      // on R: R Vj = W, sigma_i = ||w_i||, so A Q2 = (Q_C W Sigma^{-1}) Sigma Vj^T.
      double* Q2 = w.q.Y;
      QDWHP_TRY(orgqr_columns(st, w.f, ind, ell, Q2, n, w.qr_scratch));
      // Optional FP64 subspace iteration on Q2 (not in the paper): the components of the wanted
      // right singular vectors outside span(Q2) shrink by (sigma_out / sigma_k)^2 per step.
      for (int r = 0; r < o.refine_steps; ++r) {
        QDWHP_TRY(gemm(st, false, false, m, ell, n, 1.0, A, lda, Q2, n, 0.0, w.C, m));
        QDWHP_TRY(gemm(st, true, false, n, ell, m, 1.0, A, lda, w.C, m, 0.0, w.X, n));
        QDWHP_TRY(orth(st, n, ell, w.X, Q2, w.f, w.qr_scratch));
      }
      QDWHP_TRY(gemm(st, false, false, m, ell, n, 1.0, A, lda, Q2, n, 0.0, w.C, m));
      QDWHP_TRY(geqrf(st, m, ell, w.C, m, w.q.qf, w.q.qr_scratch));
      QDWHP_TRY(copy_upper(st, ell, w.C, m, w.W, ell));
      rr_unit = ell > kSvdJacobiMax && w.rr != nullptr;
      if (rr_unit) {
        // R = U_R Sigma V_R^T by QDWH-SVD: W := U_R (unit columns), Vj := V_R, vals := sigma
        QDWHP_TRY(gesvd_square(st, ell, w.W, ell, w.c.vals, w.W, ell, w.Vj, ell, w.rr, w.rr_bytes, &sweeps));
      } else {
        QDWHP_TRY(jacobi_onesided(st, ell, ell, w.W, ell, w.Vj, ell, o.jacobi_max_sweeps, kJacobiTight, w.c.jst,
                                  &hs.jst, &sweeps, &conv));
        if (!conv) return QDWHP_ERR_NOT_CONVERGED;
        QDWHP_TRY(column_norms(st, ell, ell, w.W, ell, w.c.vals));
      }
      inf.jacobi_sweeps = sweeps;
      // Step 7: sigma >= s alpha, descending.
      QDWHP_TRY(select_sort(st, ell, w.c.vals, -1.0, -s * alpha, w.c.order, w.c.ints + 1));
      QDWHP_TRY(sync_read(st, hs.ints, w.c.ints, sizeof(int) * 4));
      count = hs.ints[1];
    }
    if (count >= k || retries >= o.max_retries) break;
    ++retries;
    s = std::max(0.5 * s, 1e-15);
  }
  if (count < k) return QDWHP_ERR_COUNT;
  // Step 8: U1 = Q_C [W_sel Sigma_sel^{-1}; 0] with the Jacobi-rotated columns of R (which
  // stay orthogonal to high relative accuracy even for small sigma), or Q_C [U_R,sel; 0] from
  // QDWH-SVD; V1 = Q2 V~1 with the selected columns rescaled to unit norm (rotation rounding
  // drifts their norms).
  double* Vsel = w.X;               // ell x k
  QDWHP_TRY(gather_values(st, k, w.c.vals, w.c.order, sigma));
  QDWHP_TRY(gather_columns(st, ell, k, w.W, ell, w.c.order, rr_unit ? nullptr : w.c.vals, U, ldu));
  if (m > ell) QDWHP_TRY(set_matrix(st, m - ell, k, 0.0, 0.0, U + ell, ldu));
  QDWHP_TRY(ormqr_left(st, w.q.qf, U, k, ldu, w.q.qr_scratch));
  QDWHP_TRY(gather_columns(st, ell, k, w.Vj, ell, w.c.order, nullptr, Vsel, ell));
  QDWHP_TRY(normalize_columns(st, ell, k, Vsel, ell, nullptr));
  QDWHP_TRY(gemm(st, false, false, n, k, ell, 1.0, w.q.Y, n, Vsel, ell, 0.0, V, ldv));
  inf.ms_total = timer.stop();
  inf.retries = retries;
  inf.ell = ell;
  inf.k = k;
  inf.s = s;
  inf.alpha = alpha;
  if (info) *info = inf;
  return QDWHP_OK;
}

bool opts_valid(const qdwhp_opts& o) {
  return o.s_eig > 0.0 && o.s_eig < 1.0 && o.iters_eig >= 1 && o.iters_eig <= kMaxSteps && o.tol > 0.0 &&
         o.c_qr > 0.0 && o.block_extra >= 0 && o.power_steps >= 0 && o.power_steps <= 16 && o.lanczos_steps >= 1 &&
         o.guard >= 0.0 && o.guard < 1.0 && o.max_retries >= 0 && o.jacobi_max_sweeps >= 1 &&
         o.refine_steps >= 0 && o.refine_steps <= 64 && o.zolo_r >= 0 && o.zolo_r <= kZoloMaxR &&
         (o.use_omega == 0 || o.use_omega == 1) && o.zolo_c_qr > 0.0 &&
         (o.zolo_r == 0 || o.precision == QDWHP_FP64 || o.precision == QDWHP_FP64_EMULATED) &&
         (o.side == QDWHP_LARGEST || o.side == QDWHP_SMALLEST) &&
         (o.precision == QDWHP_FP64 || o.precision == QDWHP_MIXED || o.precision == QDWHP_FP64_EMULATED ||
          o.precision == QDWHP_MIXED_EMULATED);
}

}  // namespace
}  // namespace qdwhp

using namespace qdwhp;

extern "C" {

QDWHP_API void qdwhp_default_opts(qdwhp_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->count = 0;
  o->fraction = 0.1;
  o->side = QDWHP_LARGEST;
  o->precision = QDWHP_FP64;
  o->s_eig = 0.2;
  o->iters_eig = 3;
  o->lanczos_steps = 30;
  o->tol = 0.1;
  o->c_qr = 100.0;
  o->block_extra = 16;
  o->power_steps = 0;   // automatic: 6 for EIG, 2 for SVD
  o->guard = 0.10;
  o->max_retries = 2;
  o->jacobi_max_sweeps = 30;
  o->seed = 1234;
  o->refine_steps = 0;
  o->zolo_r = 0;
  o->use_omega = 0;
  o->zolo_c_qr = 20.0;
}

QDWHP_API const char* qdwhp_status_string(qdwhp_status s) {
  switch (s) {
    case QDWHP_OK: return "ok";
    case QDWHP_ERR_ARG: return "invalid argument";
    case QDWHP_ERR_NOMEM: return "workspace too small";
    case QDWHP_ERR_NOT_CONVERGED: return "reduced-problem Jacobi solver did not converge";
    case QDWHP_ERR_BREAKDOWN: return "Cholesky breakdown (non-positive pivot)";
    case QDWHP_ERR_NONFINITE: return "non-finite input or intermediate";
    case QDWHP_ERR_TIMEOUT: return "bounded wait expired";
    case QDWHP_ERR_CUDA: return "CUDA runtime error";
    case QDWHP_ERR_QUEUE_FULL: return "request queue full";
    case QDWHP_ERR_COUNT: return "fewer than k wanted pairs captured";
    case QDWHP_PENDING: return "pending";
  }
  return "unknown status";
}

QDWHP_API const char* qdwhp_last_error_message(void) { return g_err; }

QDWHP_API int64_t qdwhp_k_from_fraction(int64_t n, double fraction) {
  if (n < 1 || !(fraction > 0.0)) return 0;
  double kf = std::ceil(fraction * (double)n - 1e-9);
  int64_t k = (int64_t)kf;
  return std::max<int64_t>(1, std::min<int64_t>(n, k));
}

QDWHP_API size_t qdwhp_eig_workspace_bytes(int64_t n, const qdwhp_opts* opts) {
  qdwhp_opts o;
  if (opts) o = *opts; else qdwhp_default_opts(&o);
  if (n < 1) return 0;
  Arena ar;
  ar.dry = true;
  EigWs w;
  carve_eig(ar, n, o, w);
  return ar.used;
}

QDWHP_API qdwhp_status qdwhp_eig(const double* A, int64_t n, int64_t lda, const qdwhp_opts* opts, double* lambda,
                                 double* V, int64_t ldv, void* workspace, size_t ws_bytes, qdwhp_info* info,
                                 void* stream) {
  if (!opts || !A || !lambda || !V || n < 1 || lda < n || ldv < n) return QDWHP_ERR_ARG;
  if (!opts_valid(*opts)) return QDWHP_ERR_ARG;
  if (n > (1 << 20)) return QDWHP_ERR_ARG;
  if (!workspace || ws_bytes < qdwhp_eig_workspace_bytes(n, opts)) return QDWHP_ERR_NOMEM;
  return eig_impl(A, n, lda, *opts, lambda, V, ldv, workspace, ws_bytes, info, (cudaStream_t)stream);
}

QDWHP_API size_t qdwhp_svd_workspace_bytes(int64_t m, int64_t n, const qdwhp_opts* opts) {
  qdwhp_opts o;
  if (opts) o = *opts; else qdwhp_default_opts(&o);
  if (m < 1 || n < 1) return 0;
  Arena ar;
  ar.dry = true;
  SvdWs w;
  carve_svd(ar, std::max(m, n), std::min(m, n), o, w, m < n);
  return ar.used;
}

QDWHP_API qdwhp_status qdwhp_svd(const double* A, int64_t m, int64_t n, int64_t lda, int64_t k,
                                 const qdwhp_opts* opts, double* sigma, double* U, int64_t ldu, double* V,
                                 int64_t ldv, void* workspace, size_t ws_bytes, qdwhp_info* info, void* stream) {
  if (!opts || !A || !sigma || !U || !V || m < 1 || n < 1 || lda < m || ldu < m || ldv < n) return QDWHP_ERR_ARG;
  if (!opts_valid(*opts) || k < 0) return QDWHP_ERR_ARG;
  const int64_t mm = std::max(m, n), nn = std::min(m, n);
  const int64_t kk = resolve_k(nn, *opts, k);
  if (kk < 1 || kk > nn) return QDWHP_ERR_ARG;
  if (mm > (1 << 20)) return QDWHP_ERR_ARG;
  if (!workspace || ws_bytes < qdwhp_svd_workspace_bytes(m, n, opts)) return QDWHP_ERR_NOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar{(char*)workspace, ws_bytes};
  SvdWs w;
  carve_svd(ar, mm, nn, *opts, w, m < n);
  if (!ar.ok()) return QDWHP_ERR_NOMEM;
  EmulationScope emu_scope(w.emu, w.emu_bytes);
  Fp32TensorScope f32_scope(w.f32tc, w.f32tc_bytes);
  if (m >= n) return svd_impl(A, m, n, lda, kk, *opts, sigma, U, ldu, V, ldv, w, info, st);
  // m < n: solve on A^T (n x m) and swap the roles of U and V (Section 4.2).
  QDWHP_TRY(transpose(st, m, n, A, lda, w.At, n));
  return svd_impl(w.At, n, m, n, kk, *opts, sigma, V, ldv, U, ldu, w, info, st);
}

// ---- host-buffer forms: the copies run on the caller's stream inside the library ----

namespace {
struct HostIo {
  double* A = nullptr;
  double* vals = nullptr;
  double* U = nullptr;
  double* V = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
};

// Device copies of the input and outputs in front of the solver's own workspace.
void carve_host_io(Arena& ar, int64_t m, int64_t n, int64_t k, bool svd, HostIo& h) {
  h.A = ar.take<double>((size_t)m * n);
  h.vals = ar.take<double>((size_t)k);
  if (svd) h.U = ar.take<double>((size_t)m * k);
  h.V = ar.take<double>((size_t)n * k);
  const size_t front = ar.used;
  h.ws = ar.take<char>(0);
  h.ws_bytes = ar.cap > front ? ar.cap - front : 0;
}

qdwhp_status copy_in(cudaStream_t st, double* dst, const double* src_host, int64_t rows, int64_t cols, int64_t ld) {
  QDWHP_CUDA_TRY(cudaMemcpy2DAsync(dst, rows * sizeof(double), src_host, ld * sizeof(double), rows * sizeof(double),
                                   cols, cudaMemcpyHostToDevice, st));
  return QDWHP_OK;
}

qdwhp_status copy_out(cudaStream_t st, double* dst_host, int64_t ld, const double* src, int64_t rows, int64_t cols) {
  QDWHP_CUDA_TRY(cudaMemcpy2DAsync(dst_host, ld * sizeof(double), src, rows * sizeof(double), rows * sizeof(double),
                                   cols, cudaMemcpyDeviceToHost, st));
  return QDWHP_OK;
}
}  // namespace

QDWHP_API size_t qdwhp_eig_host_workspace_bytes(int64_t n, const qdwhp_opts* opts) {
  qdwhp_opts o;
  if (opts) o = *opts; else qdwhp_default_opts(&o);
  const int64_t k = resolve_k(n, o, 0);
  if (n < 1 || k < 1 || k > n) return 0;
  Arena ar;
  ar.dry = true;
  HostIo h;
  carve_host_io(ar, n, n, k, false, h);
  return ar.used + qdwhp_eig_workspace_bytes(n, &o) + 256;
}

QDWHP_API qdwhp_status qdwhp_eig_host(const double* A_host, int64_t n, int64_t lda, const qdwhp_opts* opts,
                                      double* lambda_host, double* V_host, int64_t ldv, void* workspace,
                                      size_t ws_bytes, qdwhp_info* info, void* stream) {
  if (!opts || !A_host || !lambda_host || !V_host || n < 1 || lda < n || ldv < n) return QDWHP_ERR_ARG;
  if (!opts_valid(*opts) || n > (1 << 20)) return QDWHP_ERR_ARG;
  const int64_t k = resolve_k(n, *opts, 0);
  if (k < 1 || k > n) return QDWHP_ERR_ARG;
  if (!workspace || ws_bytes < qdwhp_eig_host_workspace_bytes(n, opts)) return QDWHP_ERR_NOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar{(char*)workspace, ws_bytes};
  HostIo h;
  carve_host_io(ar, n, n, k, false, h);
  QDWHP_TRY(copy_in(st, h.A, A_host, n, n, lda));
  QDWHP_TRY(qdwhp_eig(h.A, n, n, opts, h.vals, h.V, n, h.ws, h.ws_bytes, info, stream));
  QDWHP_CUDA_TRY(cudaMemcpyAsync(lambda_host, h.vals, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
  QDWHP_TRY(copy_out(st, V_host, ldv, h.V, n, k));
  QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  return QDWHP_OK;
}

QDWHP_API size_t qdwhp_svd_host_workspace_bytes(int64_t m, int64_t n, int64_t k, const qdwhp_opts* opts) {
  qdwhp_opts o;
  if (opts) o = *opts; else qdwhp_default_opts(&o);
  if (m < 1 || n < 1) return 0;
  const int64_t kk = resolve_k(std::min(m, n), o, k);
  if (kk < 1 || kk > std::min(m, n)) return 0;
  Arena ar;
  ar.dry = true;
  HostIo h;
  carve_host_io(ar, m, n, kk, true, h);
  return ar.used + qdwhp_svd_workspace_bytes(m, n, &o) + 256;
}

QDWHP_API qdwhp_status qdwhp_svd_host(const double* A_host, int64_t m, int64_t n, int64_t lda, int64_t k,
                                      const qdwhp_opts* opts, double* sigma_host, double* U_host, int64_t ldu,
                                      double* V_host, int64_t ldv, void* workspace, size_t ws_bytes,
                                      qdwhp_info* info, void* stream) {
  if (!opts || !A_host || !sigma_host || !U_host || !V_host || m < 1 || n < 1 || lda < m || ldu < m || ldv < n)
    return QDWHP_ERR_ARG;
  if (!opts_valid(*opts) || k < 0 || std::max(m, n) > (1 << 20)) return QDWHP_ERR_ARG;
  const int64_t kk = resolve_k(std::min(m, n), *opts, k);
  if (kk < 1 || kk > std::min(m, n)) return QDWHP_ERR_ARG;
  if (!workspace || ws_bytes < qdwhp_svd_host_workspace_bytes(m, n, k, opts)) return QDWHP_ERR_NOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar{(char*)workspace, ws_bytes};
  HostIo h;
  carve_host_io(ar, m, n, kk, true, h);
  QDWHP_TRY(copy_in(st, h.A, A_host, m, n, lda));
  QDWHP_TRY(qdwhp_svd(h.A, m, n, m, kk, opts, h.vals, h.U, m, h.V, n, h.ws, h.ws_bytes, info, stream));
  QDWHP_CUDA_TRY(cudaMemcpyAsync(sigma_host, h.vals, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
  QDWHP_TRY(copy_out(st, U_host, ldu, h.U, m, kk));
  QDWHP_TRY(copy_out(st, V_host, ldv, h.V, n, kk));
  QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  return QDWHP_OK;
}

}  // extern "C"
