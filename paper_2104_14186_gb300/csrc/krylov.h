// Internal interfaces of krylov.cu and jacobi.cu.
#pragma once

#include "internal.h"

namespace qdwhp {

struct LanczosState {
  double alpha[64];
  double beta[64];
  int m;              // steps taken (set at the end or at a breakdown)
  int nonfinite;
  double out[4];      // theta_min, res_min, theta_max, res_max
};

qdwhp_status gemv_t(cudaStream_t st, int64_t m, int64_t n, const double* A, int64_t lda, const double* x, double* y);
size_t gemv_n_part_elems(int64_t m, int64_t n);
qdwhp_status gemv_n(cudaStream_t st, int64_t m, int64_t n, const double* A, int64_t lda, const double* x, double* y,
                    double* part);
qdwhp_status fill_uniform(cudaStream_t st, int64_t rows, int64_t cols, uint64_t seed, double* out, int64_t ld);
// rows x cols block of N(0, scale^2) samples (SplitMix64 + Box-Muller, column-major order).
qdwhp_status fill_gaussian(cudaStream_t st, int64_t rows, int64_t cols, uint64_t seed, double scale, double* out,
                           int64_t ld);
size_t lanczos_ws_elems(int64_t m, int64_t n, int steps);
// normal == false: symmetric n x n A; normal == true: the operator A^T A of the m x n A.
qdwhp_status lanczos(cudaStream_t st, bool normal, int64_t m, int64_t n, const double* A, int64_t lda, int steps,
                     uint64_t seed, double* ws, LanczosState* stt);
// Split point near the median of the spectrum from the Gauss quadrature of the tridiagonal
// a lanczos() run left in *stt (device): out_dev[0] = the point, out_dev[1] = the predicted
// fraction of eigenvalues at or below it, -1 if no estimate.
qdwhp_status quadrature_median(cudaStream_t st, const LanczosState* stt, double* out_dev);
// Stochastic Lanczos quadrature threshold from `probes` (<= 16) Lanczos runs on A (states, device):
// out_dev[0] = the smallest Gauss node x of A' = eps A at which n (mean lower bound of the probes'
// spectral distributions - z stderr) >= k, out_dev[1] = 1; out_dev[1] = 0 if none qualifies.
qdwhp_status slq_threshold(cudaStream_t st, const LanczosState* states, int probes, double eps, int64_t n, int64_t k,
                           double z, double* out_dev);

// ---- jacobi.cu ----
struct JacobiState {
  unsigned long long max_off_bits;  // max over a sweep of |g_p^T g_q| / (||g_p|| ||g_q||), as double bits
  int nonfinite;
};
// One-sided (Hestenes) Jacobi on the columns of G (mg x nc): G Vj = W with orthogonal
// columns, Vj (nc x nc) orthogonal.  Runs sweeps until the largest normalised inner
// product of a sweep is <= tol (or stagnates below sqrt(mg) u) or max_sweeps;
// *sweeps_out = sweeps run, *conv_out = 1 if converged.  Synchronises the stream once
// per sweep.
qdwhp_status jacobi_onesided(cudaStream_t st, int64_t mg, int64_t nc, double* G, int64_t ldg, double* Vj,
                             int64_t ldv, int max_sweeps, double tol, JacobiState* jst_dev, JacobiState* jst_host,
                             int* sweeps_out, int* conv_out);
// Scales each column of X (rows x ncols) to unit 2-norm; norms (may be null) receives the old norms.
qdwhp_status normalize_columns(cudaStream_t st, int64_t rows, int64_t ncols, double* X, int64_t ldx, double* norms);
// norms[i] = ||G(:, i)||_2
qdwhp_status column_norms(cudaStream_t st, int64_t mg, int64_t nc, const double* G, int64_t ldg, double* norms);
// d[i] = v_i^T MV(:, i) (Rayleigh quotients from MV = M V)
qdwhp_status column_dots(cudaStream_t st, int64_t mg, int64_t nc, const double* V, int64_t ldv, const double* MV,
                         int64_t ldmv, double* d);
// Selection and ordering: keys[i] = sign * vals[i]; selected iff keys[i] <= thresh_key.
// order[r] = index of the r-th smallest selected key (ties by index); *count_dev = #selected.
qdwhp_status select_sort(cudaStream_t st, int64_t nvals, const double* vals, double sign, double thresh_key,
                         int* order, int* count_dev);
// out(:, r) = scale_r * in(:, order[r]) for r < k, scale_r = 1 or 1 / norms[order[r]].
qdwhp_status gather_columns(cudaStream_t st, int64_t rows, int64_t k, const double* in, int64_t ldin, const int* order,
                            const double* inv_scale_by, double* out, int64_t ldout);
// out[r] = vals[order[r]]
qdwhp_status gather_values(cudaStream_t st, int64_t k, const double* vals, const int* order, double* out);

}  // namespace qdwhp
