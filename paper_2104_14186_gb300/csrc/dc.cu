// Symmetric eigendecomposition by QDWH spectral divide and conquer (QDWH-EIG, Section 3.2).
//
// A node holds a symmetric matrix M (order nl) whose spectrum lies in [lo, hi].  It picks a
// split point sigma near the median of its spectrum (a midpoint of Gauss quadrature nodes of
// 30 Lanczos steps on M; then the mean eigenvalue trace / nl and the middle of [lo, hi] if a
// split is one-sided or leaves an eigenvalue unresolved), computes the polar factor U_p of
// (M - sigma I) / alpha with alpha = max(sigma - lo, hi - sigma) >= ||M - sigma I||_2 by QDWH
// (eqs. practical-polar-qr / practical-polar-chol, ell_0 = kDcEll0, so QR-based steps first),
// and forms the projector P = (I + U_p) / 2 onto the eigenvectors with eigenvalues above sigma
// (eq. pdeig and the projector identity after it).  Its rank r = trace(P).  A basis Q1 of
// range(P) comes from the Householder QR of P Omega (Omega: r SplitMix64 columns) followed by
// one subspace-iteration pass (QR of P Q1), which makes the basis accurate to working
// precision; the full orthogonal factor Q = [Q1 Q2] of that QR also supplies the complement
// Q2.  The two children are the Rayleigh-Ritz matrices M1 = Q1^T M Q1 (spectrum in
// [sigma, hi]) and M2 = Q2^T M Q2 (in [lo, sigma]); the off-diagonal block E = Q2^T M Q1 is
// the backward error of the split and is checked.  Nodes of order <= kDcLeaf are solved by
// one-sided Jacobi on M - lower I (positive semidefinite) with Rayleigh-quotient eigenvalues.
//
// Eigenvectors are accumulated in place: every node multiplies its column block of V by its
// Q (or, at a leaf, by the Jacobi vectors), so no per-level basis is kept.  Children are
// stored in their parent's slot of w.M (r^2 + (nl - r)^2 <= nl^2), so the whole recursion
// runs in the workspace of the top node.
#include <cmath>
#include <cstring>

#include "dc.h"

namespace qdwhp {

namespace {

constexpr uint64_t kStreamSplit = 0x44435350ull;   // "DCSP"
constexpr uint64_t kStreamSlq = 0x44435351ull;     // "DCSQ"
constexpr int kSlqSteps = 30;
constexpr double kUnresolved = 0.05;
constexpr double kJacobiTightDc = 4.5e-16;
constexpr double kJacobiValues = 1e-9;
constexpr int kMaxDepth = 64;

// out = sum of the diagonal of A (one CTA, fixed summation order).
__global__ void diag_sum_kernel(int n, const double* A, int64_t lda, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += A[i + (int64_t)i * lda];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) *out = acc;
}

// parts[b] = sum of squares of the entries block b visits (fixed grid, so the two-stage sum
// is deterministic).
__global__ void sumsq_parts_kernel(int m, int n, const double* A, int64_t lda, double* parts) {
  __shared__ double red[32];
  const size_t total = (size_t)m * n;
  double acc = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    const double v = A[i + (int64_t)j * lda];
    acc = fma(v, v, acc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) parts[blockIdx.x] = acc;
}

qdwhp_status read_scalar(cudaStream_t st, const double* dev, double* host) {
  QDWHP_CUDA_TRY(cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  return QDWHP_OK;
}

struct Ctx {
  cudaStream_t st;
  int64_t n;                 // order of the top problem (rows of V)
  uint64_t seed;
  bool vectors;
  int max_sweeps;
  double* lam;
  double* V;
  int64_t ldv;
  DcWs* w;
  DcStats* stats;
  double scale;              // max(|lo|, |hi|) of the top problem
  Schedule sched;            // the polar schedule from kDcEll0 (the same at every node)
  JacobiState jst_host;
  int node_counter = 0;
};

// V(:, c0 : c0 + nl) := V(:, c0 : c0 + nl) B, B nl x nl (ld nl), through w.W.
qdwhp_status update_vectors(Ctx& c, int64_t c0, int64_t nl, const double* B) {
  double* Vb = c.V + c0 * c.ldv;
  QDWHP_TRY(gemm(c.st, false, false, c.n, nl, nl, 1.0, Vb, c.ldv, B, nl, 0.0, c.w->W, c.n));
  return copy_matrix(c.st, c.n, nl, c.w->W, c.n, Vb, c.ldv);
}

// Leaf: one-sided Jacobi on G = M - lower I; eigenvalues are the Rayleigh quotients.
qdwhp_status leaf(Ctx& c, int64_t c0, int64_t nl, size_t moff, double lo, double hi) {
  DcWs& w = *c.w;
  double* Mn = w.M + moff;
  c.stats->leaves += 1;
  if (nl == 1) {
    QDWHP_TRY(copy_matrix(c.st, 1, 1, Mn, 1, c.lam + c0, 1));
    return QDWHP_OK;   // V's column is already the eigenvector
  }
  // lower <= lambda_min(Mn), with a margin for the backward error of the splits above
  const double lower = lo - 0.01 * (hi - lo) - 1e-12 * c.scale;
  QDWHP_TRY(axpby(c.st, nl, nl, 1.0, Mn, nl, 0.0, w.W, nl, -lower));
  int sweeps = 0, conv = 0;
  const double tol = c.vectors ? kJacobiTightDc : kJacobiValues;
  QDWHP_TRY(jacobi_onesided(c.st, nl, nl, w.W, nl, w.Q, nl, c.max_sweeps, tol, w.jst, &c.jst_host, &sweeps, &conv));
  if (!conv) return QDWHP_ERR_NOT_CONVERGED;
  c.stats->jacobi_sweeps = std::max(c.stats->jacobi_sweeps, sweeps);
  QDWHP_TRY(normalize_columns(c.st, nl, nl, w.Q, nl, nullptr));
  QDWHP_TRY(gemm(c.st, false, false, nl, nl, nl, 1.0, Mn, nl, w.Q, nl, 0.0, w.X, nl));
  QDWHP_TRY(column_dots(c.st, nl, nl, w.Q, nl, w.X, nl, c.lam + c0));
  if (c.vectors) QDWHP_TRY(update_vectors(c, c0, nl, w.Q));
  return QDWHP_OK;
}

// Q (nl x nl) := full orthogonal factor of the Householder QR of Y (nl x r, in w.W).
qdwhp_status split_basis(Ctx& c, int64_t nl, int64_t r) {
  DcWs& w = *c.w;
  QDWHP_TRY(geqrf(c.st, nl, r, w.W, nl, w.f, w.qr_scratch));
  QDWHP_TRY(set_matrix(c.st, nl, nl, 0.0, 1.0, w.Q, nl));
  return ormqr_left(c.st, w.f, w.Q, nl, nl, w.qr_scratch);
}

qdwhp_status node(Ctx& c, int64_t c0, int64_t nl, size_t moff, double lo, double hi, int depth) {
  DcWs& w = *c.w;
  cudaStream_t st = c.st;
  double* Mn = w.M + moff;
  // a leaf, a (numerically) single point, or a runaway recursion: Jacobi
  if (nl <= kDcLeaf || hi - lo <= 1e-14 * c.scale || depth >= kMaxDepth) return leaf(c, c0, nl, moff, lo, hi);

  // Split point: near the median of the spectrum, from the Gauss quadrature of a short
  // Lanczos run on M (Golub-Welsch), so that graded spectra split evenly.  A candidate is
  // kept when its split is two-sided and resolved: P = (I + U_p) / 2 is a projector to
  // rounding, trace(P) - ||P||_F^2 = sum p (1 - p) <= kUnresolved (an eigenvalue within the
  // polar resolution ell_0 of sigma gives p ~ 1/2).  Otherwise the next candidate: the mean
  // eigenvalue trace(M) / nl, then the middle of [lo, hi].
  const uint64_t slq_seed = c.seed ^ kStreamSlq ^ ((uint64_t)(c.node_counter + 1) * 0xD1B54A32D192ED03ull);
  QDWHP_TRY(lanczos(st, false, nl, nl, Mn, nl, kSlqSteps, slq_seed, w.lws, w.lst));
  QDWHP_TRY(quadrature_median(st, w.lst, w.scal + 4));
  diag_sum_kernel<<<1, 1024, 0, st>>>((int)nl, Mn, nl, w.scal);
  QDWHP_LAUNCH_CHECK();
  double sc[6];
  QDWHP_CUDA_TRY(cudaMemcpyAsync(sc, w.scal, sizeof(sc), cudaMemcpyDeviceToHost, st));
  QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  double cand[3];
  int ncand = 0;
  const bool have_median = sc[5] > 0.0 && std::isfinite(sc[4]);
  if (have_median) cand[ncand++] = sc[4];
  cand[ncand++] = sc[0] / (double)nl;
  cand[ncand++] = 0.5 * (lo + hi);
  double sigma = 0.0, alpha = 0.0;
  int64_t r = 0;
  for (int ci = 0; ci < ncand; ++ci) {
    sigma = std::min(std::max(cand[ci], lo), hi);
    alpha = std::max(sigma - lo, hi - sigma) + 1e-12 * c.scale;
    // polar factor of (M - sigma I) / alpha
    QDWHP_TRY(axpby(st, nl, nl, 1.0 / alpha, Mn, nl, 0.0, w.X, nl, -sigma / alpha));
    QDWHP_CUDA_TRY(cudaMemsetAsync(w.q.fail, 0, sizeof(int), st));
    int n_qr = 0, n_chol = 0, n_f32 = 0;
    QDWHP_TRY(run_schedule(st, nl, nl, w.X, nl, c.sched, false, w.q, &n_qr, &n_chol, &n_f32));
    c.stats->qdwh_steps += n_qr + n_chol;
    // P = (I + U_p) / 2, symmetrised
    QDWHP_TRY(symmetrize_avg(st, nl, w.X, nl));
    QDWHP_TRY(axpby(st, nl, nl, 0.5, w.X, nl, 0.0, w.X, nl, 0.5));
    diag_sum_kernel<<<1, 1024, 0, st>>>((int)nl, w.X, nl, w.scal + 1);
    QDWHP_LAUNCH_CHECK();
    int fail = 0;
    QDWHP_CUDA_TRY(cudaMemcpyAsync(&fail, w.q.fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    double trP = 0.0;
    QDWHP_TRY(read_scalar(st, w.scal + 1, &trP));
    if (fail) return QDWHP_ERR_BREAKDOWN;
    if (!std::isfinite(trP)) return QDWHP_ERR_NONFINITE;
    r = std::min<int64_t>(nl, std::max<int64_t>(0, std::llround(trP)));
    if (r > 0 && r < nl) {
      sumsq_parts_kernel<<<kDiffParts, 256, 0, st>>>((int)nl, (int)nl, w.X, nl, w.parts);
      QDWHP_LAUNCH_CHECK();
      QDWHP_TRY(reduce_parts(st, w.parts, kDiffParts, w.scal + 3));
      double p2 = 0.0;
      QDWHP_TRY(read_scalar(st, w.scal + 3, &p2));
      if (!std::isfinite(p2)) return QDWHP_ERR_NONFINITE;
      if (trP - p2 <= kUnresolved) {
        if (ci == 0 && have_median) c.stats->median_splits += 1;
        break;
      }
      c.stats->unresolved_splits += 1;
    }
    r = 0;
  }
  // No candidate split two-sidedly and resolved: the eigenvalues lie within the polar
  // resolution of every candidate, a cluster, which Jacobi settles at once.
  if (r == 0 || r == nl) return leaf(c, c0, nl, moff, lo, hi);
  c.stats->nodes += 1;
  c.stats->depth = std::max(c.stats->depth, depth + 1);

  // Q1: range of P Omega, then one subspace-iteration pass P Q1.
  const uint64_t node_seed = c.seed ^ kStreamSplit ^ ((uint64_t)(++c.node_counter) * 0x9E3779B97F4A7C15ull);
  QDWHP_TRY(fill_uniform(st, nl, r, node_seed, w.Q, nl));
  QDWHP_TRY(gemm(st, false, false, nl, r, nl, 1.0, w.X, nl, w.Q, nl, 0.0, w.W, nl));
  QDWHP_TRY(split_basis(c, nl, r));
  double off = INFINITY;
  for (int pass = 0; pass < 3; ++pass) {
    QDWHP_TRY(gemm(st, false, false, nl, r, nl, 1.0, w.X, nl, w.Q, nl, 0.0, w.W, nl));
    QDWHP_TRY(split_basis(c, nl, r));
    // W = M Q;  E = Q2^T (M Q1), ||E||_F
    QDWHP_TRY(gemm(st, false, false, nl, nl, nl, 1.0, Mn, nl, w.Q, nl, 0.0, w.W, nl));
    QDWHP_TRY(gemm(st, true, false, nl - r, r, nl, 1.0, w.Q + r * nl, nl, w.W, nl, 0.0, w.E, nl - r));
    sumsq_parts_kernel<<<kDiffParts, 256, 0, st>>>((int)(nl - r), (int)r, w.E, nl - r, w.parts);
    QDWHP_LAUNCH_CHECK();
    QDWHP_TRY(reduce_parts(st, w.parts, kDiffParts, w.scal + 2));
    double e2 = 0.0;
    QDWHP_TRY(read_scalar(st, w.scal + 2, &e2));
    if (!std::isfinite(e2)) return QDWHP_ERR_NONFINITE;
    off = std::sqrt(e2) / alpha;
    // backward error of the split at the level of the rounding of the products
    if (off <= 64.0 * 2.220446049250313e-16 * std::sqrt((double)nl)) break;
    c.stats->refinements += 1;
  }
  c.stats->max_offblock = std::max(c.stats->max_offblock, off);

  // children: M1 = Q1^T (M Q1) (r x r) and M2 = Q2^T (M Q2) into this node's slot
  QDWHP_TRY(gemm(st, true, false, r, r, nl, 1.0, w.Q, nl, w.W, nl, 0.0, Mn, r));
  QDWHP_TRY(gemm(st, true, false, nl - r, nl - r, nl, 1.0, w.Q + r * nl, nl, w.W + r * nl, nl, 0.0,
                 Mn + (size_t)r * r, nl - r));
  QDWHP_TRY(symmetrize_avg(st, r, Mn, r));
  QDWHP_TRY(symmetrize_avg(st, nl - r, Mn + (size_t)r * r, nl - r));
  if (c.vectors) {
    if (depth == 0) {
      QDWHP_TRY(copy_matrix(st, nl, nl, w.Q, nl, c.V + c0 * c.ldv, c.ldv));   // V = I Q
    } else {
      QDWHP_TRY(update_vectors(c, c0, nl, w.Q));
    }
  }
  QDWHP_TRY(node(c, c0, r, moff, sigma, hi, depth + 1));
  return node(c, c0 + r, nl - r, moff + (size_t)r * r, lo, sigma, depth + 1);
}

}  // namespace

void carve_dc_own(Arena& ar, int64_t cap, DcWs& w) {
  const size_t c2 = (size_t)cap * cap;
  w.cap = cap;
  w.E = ar.take<double>(c2 / 4 + cap + 64);
  carve_qdwh(ar, cap, cap, true, w.q, false);
  w.sched = ar.take<Schedule>(1);
  w.scal = ar.take<double>(8);
  w.parts = ar.take<double>(kDiffParts);
  w.jst = ar.take<JacobiState>(1);
  w.lst = ar.take<LanczosState>(1);
  w.lws = ar.take<double>(lanczos_ws_elems(cap, cap, kSlqSteps));
}

void carve_dc(Arena& ar, int64_t cap, DcWs& w) {
  const size_t c2 = (size_t)cap * cap;
  w.M = ar.take<double>(c2);
  w.X = ar.take<double>(c2);
  w.Q = ar.take<double>(c2);
  w.W = ar.take<double>(c2);
  w.f.Vall = ar.take<double>(c2);
  w.f.T = ar.take<double>((size_t)ceil_div(cap, kQRNB) * kQRNB * kQRNB);
  w.f.To = ar.take<double>(qr_to_elems(cap));
  w.f.tau = ar.take<double>(cap);
  w.f.diagR = ar.take<double>(cap);
  w.qr_scratch = ar.take<double>(qr_scratch_elems(cap, cap));
  carve_dc_own(ar, cap, w);
}

qdwhp_status sym_eig_dc(cudaStream_t st, int64_t n, double lo, double hi, uint64_t seed, bool vectors,
                        int jacobi_max_sweeps, double* lam, double* V, int64_t ldv, DcWs& w, DcStats* stats) {
  if (n < 1 || n > w.cap || !(lo <= hi) || (vectors && ldv < n)) return QDWHP_ERR_ARG;
  DcStats local;
  Ctx c;
  c.st = st;
  c.n = n;
  c.seed = seed;
  c.vectors = vectors;
  c.max_sweeps = jacobi_max_sweeps;
  c.lam = lam;
  c.V = V;
  c.ldv = ldv;
  c.w = &w;
  c.stats = stats ? stats : &local;
  *c.stats = DcStats();
  c.scale = std::max({std::fabs(lo), std::fabs(hi), 1e-300});
  if (n > kDcLeaf) {
    QDWHP_TRY(dwh_schedule(st, nullptr, kDcEll0, 0, 100.0, w.sched));
    QDWHP_CUDA_TRY(cudaMemcpyAsync(&c.sched, w.sched, sizeof(Schedule), cudaMemcpyDeviceToHost, st));
    QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (vectors) QDWHP_TRY(set_matrix(st, n, n, 0.0, 1.0, V, ldv));
  return node(c, 0, n, 0, lo, hi, 0);
}

namespace {

constexpr int kSyevLanczosSteps = 30;
constexpr int kSyevMaxSweeps = 30;
constexpr uint64_t kSyevSeed = 1234;

struct SyevWs {
  DcWs dc;
  LanczosState* lst = nullptr;
  double* lws = nullptr;
  unsigned* nonfinite = nullptr;
  double* lam = nullptr;   // n, unordered
  int* order = nullptr;    // n
  int* count = nullptr;
  double* V = nullptr;     // n x n, unordered columns
};

void carve_syev(Arena& ar, int64_t n, SyevWs& w) {
  carve_dc(ar, n, w.dc);
  w.lst = ar.take<LanczosState>(1);
  w.lws = ar.take<double>(lanczos_ws_elems(n, n, kSyevLanczosSteps));
  w.nonfinite = ar.take<unsigned>(4);
  w.lam = ar.take<double>(n);
  w.order = ar.take<int>(n);
  w.count = ar.take<int>(4);
  w.V = ar.take<double>((size_t)n * n);
}

qdwhp_status syev_impl(const double* A, int64_t n, int64_t lda, double* lambda, double* V, int64_t ldv,
                       void* workspace, size_t ws_bytes, qdwhp_syev_info* info, cudaStream_t st) {
  Arena ar{(char*)workspace, ws_bytes};
  SyevWs w;
  carve_syev(ar, n, w);
  if (!ar.ok()) return QDWHP_ERR_NOMEM;
  EventPair ev;
  QDWHP_CUDA_TRY(cudaEventCreate(&ev.e0));
  QDWHP_CUDA_TRY(cudaEventCreate(&ev.e1));
  QDWHP_CUDA_TRY(cudaEventRecord(ev.e0, st));
  QDWHP_CUDA_TRY(cudaMemsetAsync(w.nonfinite, 0, sizeof(unsigned), st));
  QDWHP_TRY(count_nonfinite(st, n, n, A, lda, w.nonfinite));
  unsigned nonfinite = 0;
  QDWHP_CUDA_TRY(cudaMemcpyAsync(&nonfinite, w.nonfinite, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  if (nonfinite) return QDWHP_ERR_NONFINITE;
  // spectral bounds: extreme Ritz values -/+ their residuals, pushed 1 % of the spread outwards
  QDWHP_TRY(lanczos(st, false, n, n, A, lda, kSyevLanczosSteps, kSyevSeed, w.lws, w.lst));
  LanczosState lst;
  QDWHP_CUDA_TRY(cudaMemcpyAsync(&lst, w.lst, sizeof(LanczosState), cudaMemcpyDeviceToHost, st));
  QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  if (lst.nonfinite) return QDWHP_ERR_NONFINITE;
  const double lo_raw = lst.out[0] - lst.out[1], hi_raw = lst.out[2] + lst.out[3];
  const double spread = std::max(hi_raw - lo_raw, 1e-300);
  const double lo = lo_raw - 0.01 * spread, hi = hi_raw + 0.01 * spread;
  QDWHP_TRY(copy_matrix(st, n, n, A, lda, w.dc.M, n));
  QDWHP_TRY(symmetrize_avg(st, n, w.dc.M, n));
  DcStats stats;
  QDWHP_TRY(sym_eig_dc(st, n, lo, hi, kSyevSeed, true, kSyevMaxSweeps, w.lam, w.V, n, w.dc, &stats));
  QDWHP_TRY(select_sort(st, n, w.lam, 1.0, INFINITY, w.order, w.count));
  QDWHP_TRY(gather_values(st, n, w.lam, w.order, lambda));
  QDWHP_TRY(gather_columns(st, n, n, w.V, n, w.order, nullptr, V, ldv));
  QDWHP_CUDA_TRY(cudaEventRecord(ev.e1, st));
  QDWHP_CUDA_TRY(cudaEventSynchronize(ev.e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev.e0, ev.e1);
  if (info) {
    info->nodes = stats.nodes;
    info->leaves = stats.leaves;
    info->depth = stats.depth;
    info->qdwh_steps = stats.qdwh_steps;
    info->refinements = stats.refinements;
    info->jacobi_sweeps = stats.jacobi_sweeps;
    info->max_offblock = stats.max_offblock;
    info->ms_total = ms;
    info->median_splits = stats.median_splits;
  }
  return QDWHP_OK;
}

}  // namespace

}  // namespace qdwhp

using namespace qdwhp;

extern "C" {

QDWHP_API size_t qdwhp_syev_workspace_bytes(int64_t n) {
  if (n < 1) return 0;
  Arena ar;
  ar.dry = true;
  SyevWs w;
  carve_syev(ar, n, w);
  return ar.used;
}

QDWHP_API qdwhp_status qdwhp_syev_f64(const double* A, int64_t n, int64_t lda, double* lambda, double* V,
                                      int64_t ldv, void* workspace, size_t ws_bytes, qdwhp_syev_info* info,
                                      void* stream) {
  if (!A || !lambda || !V || n < 1 || lda < n || ldv < n || n > (1 << 17)) return QDWHP_ERR_ARG;
  if (!workspace || ws_bytes < qdwhp_syev_workspace_bytes(n)) return QDWHP_ERR_NOMEM;
  return syev_impl(A, n, lda, lambda, V, ldv, workspace, ws_bytes, info, (cudaStream_t)stream);
}

}  // extern "C"
