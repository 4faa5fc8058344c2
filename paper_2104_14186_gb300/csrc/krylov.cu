// Spectral bounds by Lanczos (Algorithm 1 step 1 "a few steps of the Lanczos
// iteration"; Algorithm 2 step 1 norm estimate on A^T A), HBM-bound GEMV kernels
// and the SplitMix64 start vectors.
//
// Lanczos runs with full reorthogonalisation (classical Gram-Schmidt, twice) and
// keeps every scalar on the device: the host only enqueues the steps.  Only the
// extreme eigenpairs of the tridiagonal T (at most 64 x 64) are needed: the extreme
// Ritz values and their residual norms beta_m |s_{m,i}| are the output.
#include "internal.h"
#include "krylov.h"

namespace qdwhp {

namespace {

// y = A^T x (A m x n): one warp per column, coalesced down the column.
__global__ void gemv_t_kernel(int M, int N, const double* A, int64_t lda, const double* x, double* y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= N) return;
  const double* col = A + (int64_t)warp * lda;
  double acc = 0.0;
  for (int i = lane; i < M; i += 32) acc += col[i] * x[i];
  acc = warp_sum(acc);
  if (lane == 0) y[warp] = acc;
}

// Partial y = A x over column chunks of 64: part[chunk * M + i].
constexpr int kGemvChunk = 64;
__global__ void gemv_n_part_kernel(int M, int N, const double* A, int64_t lda, const double* x, double* part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c0 = blockIdx.y * kGemvChunk;
  if (i >= M) return;
  const int c1 = min(N, c0 + kGemvChunk);
  double acc = 0.0;
  for (int j = c0; j < c1; ++j) acc += A[i + (int64_t)j * lda] * x[j];
  part[(size_t)blockIdx.y * M + i] = acc;
}

__global__ void sum_chunks_kernel(int M, int nchunks, const double* part, double* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double acc = 0.0;
  for (int c = 0; c < nchunks; ++c) acc += part[(size_t)c * M + i];
  y[i] = acc;
}

__global__ void fill_uniform_kernel(size_t count, uint64_t seed, double* out, int64_t rows, int64_t ld) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)(e % rows), j = (int64_t)(e / rows);
    out[i + j * ld] = uniform_pm1_at(seed, e);
  }
}

// Standard normal samples by the Box-Muller transform (Box and Muller 1958) of consecutive
// SplitMix64 outputs: output 2j is sqrt(-2 log u1) cos(2 pi u2) and output 2j + 1 the same
// radius times sin(2 pi u2), with u1 = ((z_2j >> 11) + 1) 2^-53 in (0, 1] and
// u2 = (z_2j+1 >> 11) 2^-53 in [0, 1); element e of the column-major rows x cols block takes
// output e, times `scale`.
__global__ void fill_gaussian_kernel(size_t count, uint64_t seed, double scale, double* out, int64_t rows,
                                     int64_t ld) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const uint64_t pair = e >> 1;
    const uint64_t z1 = splitmix64_at(seed, 2 * pair), z2 = splitmix64_at(seed, 2 * pair + 1);
    const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = (double)(z2 >> 11) * 0x1.0p-53;
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    const int64_t i = (int64_t)(e % rows), j = (int64_t)(e / rows);
    out[i + j * ld] = scale * r * ((e & 1) ? sn : cs);
  }
}

// h[c] = Q(:, c)^T w for c < ncols (one CTA per column).
__global__ void dots_t_kernel(int n, const double* Q, int64_t ldq, const double* w, double* h) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += Q[i + (int64_t)c * ldq] * w[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) h[c] = acc;
}

// w -= Q(:, 0:ncols) h
__global__ void sub_qh_kernel(int n, int ncols, const double* Q, int64_t ldq, const double* h, double* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int c = 0; c < ncols; ++c) acc += Q[i + (int64_t)c * ldq] * h[c];
  w[i] -= acc;
}

// Step finish: alpha_j = h0[j]; beta_j = ||w||; q_{j+1} = w / beta_j.  A step after a
// breakdown (state->m already set) is a no-op.
__global__ void lanczos_finish_kernel(int n, int j, int steps, const double* h0, double* w, double* qnext,
                                      LanczosState* stt) {
  __shared__ double red[32];
  if (stt->m > 0 && stt->m <= j) return;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += w[i] * w[i];
  acc = block_sum(acc, red);
  const double beta = sqrt(acc);
  const double alpha = h0[j];
  if (threadIdx.x == 0) {
    stt->alpha[j] = alpha;
    stt->beta[j] = beta;
    if (!isfinite(beta) || !isfinite(alpha)) stt->nonfinite = 1;
  }
  const bool last = (j + 1 == steps);
  const bool breakdown = beta <= 1e-14 * fmax(fabs(alpha), 1e-300);
  if (last) {
    if (threadIdx.x == 0) stt->m = j + 1;
    return;
  }
  if (breakdown) {
    if (threadIdx.x == 0) {
      stt->m = j + 1;
      stt->beta[j] = 0.0;
    }
    return;
  }
  const double inv = 1.0 / beta;
  for (int i = threadIdx.x; i < n; i += blockDim.x) qnext[i] = w[i] * inv;
}

__global__ void normalize_kernel(int n, double* q) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += q[i] * q[i];
  acc = block_sum(acc, red);
  const double inv = acc > 0.0 ? 1.0 / sqrt(acc) : 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) q[i] *= inv;
}

// Extreme eigenpairs of the m x m Lanczos tridiagonal T (one warp).  Eigenvalues by
// multisection on Sturm counts (each lane evaluates one of 32 points of the current
// interval, so every step shrinks it 33-fold); the last component of each eigenvector
// by two steps of inverse iteration with T - x I factored as L D L^T, x just outside
// the spectrum so the factorisation is definite.  Writes theta_min, its residual norm
// beta_{m-1} |s_{m-1}|, theta_max and its residual norm.
constexpr int kMaxT = 64;

__device__ int sturm_count(const double* al, const double* be, int m, double x, double pivmin) {
  // number of eigenvalues of T below x: negative pivots of T - x I = L D L^T
  int cnt = 0;
  double d = al[0] - x;
  if (fabs(d) < pivmin) d = -pivmin;
  cnt += d < 0.0;
  for (int i = 1; i < m; ++i) {
    d = (al[i] - x) - be[i - 1] * be[i - 1] / d;
    if (fabs(d) < pivmin) d = -pivmin;
    cnt += d < 0.0;
  }
  return cnt;
}

// Find the eigenvalue where the Sturm count steps to `target` (1: smallest, m: largest).
__device__ double multisect(const double* al, const double* be, int m, double lo, double hi, int target,
                            double pivmin) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < 64; ++it) {
    const double w = hi - lo;
    if (!(w > 2.0 * 0x1.0p-52 * fmax(fabs(lo), fabs(hi)) + pivmin)) break;
    const double x = lo + w * (double)(lane + 1) / 33.0;
    const int c = sturm_count(al, be, m, x, pivmin);
    const unsigned mask = __ballot_sync(0xffffffffu, c >= target);
    const int first = mask ? __ffs(mask) - 1 : 32;
    const double xf = __shfl_sync(0xffffffffu, x, first < 32 ? first : 31);
    const double xp = __shfl_sync(0xffffffffu, x, first > 0 ? first - 1 : 0);
    if (first == 32) {
      lo = xf;                       // all 32 points below the eigenvalue
    } else {
      hi = xf;
      lo = first > 0 ? xp : lo;
    }
  }
  return 0.5 * (lo + hi);
}

// |last component| / ||y|| of the eigenvector for the eigenvalue near x (lane 0).
__device__ double last_component(const double* al, const double* be, int m, double x) {
  double l[kMaxT], d[kMaxT], y[kMaxT];
  d[0] = al[0] - x;
  for (int i = 1; i < m; ++i) {
    l[i] = be[i - 1] / d[i - 1];
    d[i] = (al[i] - x) - l[i] * be[i - 1];
  }
  for (int i = 0; i < m; ++i) y[i] = 1.0;
  for (int it = 0; it < 2; ++it) {
    for (int i = 1; i < m; ++i) y[i] -= l[i] * y[i - 1];          // L z = y
    y[m - 1] /= d[m - 1];                                          // D L^T y = z
    for (int i = m - 2; i >= 0; --i) y[i] = y[i] / d[i] - l[i + 1] * y[i + 1];
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += y[i] * y[i];
    nrm = sqrt(nrm);
    for (int i = 0; i < m; ++i) y[i] /= nrm;
  }
  return fabs(y[m - 1]);
}

__global__ void tridiag_extremes_kernel(LanczosState* stt) {
  __shared__ double al[kMaxT], be[kMaxT];
  const int lane = threadIdx.x;
  const int m = max(1, min(stt->m, kMaxT));
  for (int i = lane; i < kMaxT; i += 32) {
    al[i] = i < m ? stt->alpha[i] : 0.0;
    be[i] = i < m - 1 ? stt->beta[i] : 0.0;
  }
  __syncwarp();
  // Gershgorin interval
  double lo = INFINITY, hi = -INFINITY, scale = 0.0;
  for (int i = lane; i < m; i += 32) {
    const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i < m - 1 ? fabs(be[i]) : 0.0);
    lo = fmin(lo, al[i] - r);
    hi = fmax(hi, al[i] + r);
    scale = fmax(scale, fabs(al[i]) + r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    scale = fmax(scale, __shfl_xor_sync(0xffffffffu, scale, o));
  }
  const double pivmin = fmax(scale, 1e-300) * 0x1.0p-100;
  const double pad = fmax(scale, 1e-300) * 1e-12;
  lo -= pad;
  hi += pad;
  const double tmin = multisect(al, be, m, lo, hi, 1, pivmin);
  const double tmax = multisect(al, be, m, lo, hi, m, pivmin);
  if (lane == 0) {
    const double bm = fabs(stt->beta[m - 1]);
    const double shift = fmax(scale, 1e-300) * 1e-13;
    // beta_{m-1} = 0 (an invariant subspace, e.g. a one-point spectrum): the Ritz values are
    // exact, and the eigenvector estimate is not needed (for T = 0 it would divide by ~0)
    stt->out[0] = tmin;
    stt->out[1] = bm > 0.0 ? bm * last_component(al, be, m, tmin - shift) : 0.0;
    stt->out[2] = tmax;
    stt->out[3] = bm > 0.0 ? bm * last_component(al, be, m, tmax + shift) : 0.0;
  }
}

inline int grid1d(size_t total, int threads) {
  return (int)std::max<size_t>(1, std::min<size_t>((total + threads - 1) / threads, 16 * (size_t)kNumSMs));
}

// Split point of a spectrum from the Gauss quadrature of the Lanczos tridiagonal T
// (Golub-Welsch: the nodes are the eigenvalues of T, the weights the squared first
// components of its eigenvectors), which approximates the spectral distribution of the
// operator seen from the start vector.  One thread: implicit symmetric tridiagonal QR with
// the Wilkinson shift (Golub and Van Loan, Section 8.3), accumulating only the first row of
// the eigenvector matrix.  With the nodes ascending and c_j the cumulative weights, j* is the
// first node with c_j >= 1/2.  Ritz values converge onto clusters, so a node may coincide
// with an eigenvalue; the candidates are therefore midpoints beside theta_j*, between it and
// the nearest nodes below and above that differ from it by more than 1e-8 of the nodes'
// scale (a, predicted fraction at or below: c_a; b, predicted c_{b-1}).
// out[0] = the candidate whose prediction is nearer 1/2 among those strictly inside (0, 1),
// out[1] = its prediction, or -1 when there is none (or T is not finite).
// Gauss rule of the Lanczos tridiagonal in *stt (Golub and Welsch 1969): the nodes are the
// eigenvalues of T, the weights the squared first components of its eigenvectors.  One thread:
// implicit symmetric tridiagonal QR with the Wilkinson shift (Golub and Van Loan, Section 8.3),
// accumulating only the first row of the eigenvector matrix.  On return d[0..m) holds the nodes
// ascending and z their weights normalised to sum 1; false if T is not finite, the QR did not
// converge or the weights are degenerate.
__device__ bool gauss_rule_thread(const LanczosState* stt, double* d, double* z, int* m_out) {
  if (stt->nonfinite) return false;
  const int m = max(1, min(stt->m, kMaxT));
  double e[kMaxT];
  for (int i = 0; i < m; ++i) {
    d[i] = stt->alpha[i];
    e[i] = i + 1 < m ? stt->beta[i] : 0.0;
    z[i] = i == 0 ? 1.0 : 0.0;
  }
  const double eps = 0x1.0p-52;
  int hi = m - 1;
  for (int it = 0; hi > 0 && it < 30 * kMaxT; ++it) {
    if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) --lo;
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer d[hi]
    const double dd = 0.5 * (d[hi - 1] - d[hi]), b2 = e[hi - 1] * e[hi - 1];
    const double mu = d[hi] - b2 / (dd + copysign(sqrt(dd * dd + b2), dd >= 0.0 ? 1.0 : -1.0));
    double x = d[lo] - mu, y = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = hypot(x, y);
      const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? y / r : 0.0;
      if (k > lo) e[k - 1] = r;
      const double a = d[k], b = e[k], cc = d[k + 1];
      d[k] = c * c * a + 2.0 * c * s * b + s * s * cc;
      d[k + 1] = s * s * a - 2.0 * c * s * b + c * c * cc;
      e[k] = c * s * (cc - a) + (c * c - s * s) * b;
      if (k + 1 < hi) {
        x = e[k];
        y = s * e[k + 1];   // the bulge at (k, k + 2)
        e[k + 1] *= c;
      }
      const double zk = z[k];
      z[k] = c * zk + s * z[k + 1];
      z[k + 1] = -s * zk + c * z[k + 1];
    }
  }
  if (hi > 0) return false;   // not converged: no rule
  // nodes ascending with their weights
  double wsum = 0.0;
  for (int i = 0; i < m; ++i) {
    z[i] *= z[i];
    wsum += z[i];
  }
  for (int i = 1; i < m; ++i) {
    const double di = d[i], zi = z[i];
    int j = i - 1;
    for (; j >= 0 && d[j] > di; --j) {
      d[j + 1] = d[j];
      z[j + 1] = z[j];
    }
    d[j + 1] = di;
    z[j + 1] = zi;
  }
  if (!(wsum > 0.0) || !isfinite(wsum)) return false;
  for (int i = 0; i < m; ++i) z[i] /= wsum;
  *m_out = m;
  return true;
}

// Split point of a spectrum from the Gauss quadrature of the Lanczos tridiagonal T, which
// approximates the spectral distribution of the operator seen from the start vector.  With
// the nodes ascending and c_j the cumulative weights, j* is the first node with c_j >= 1/2.
// Ritz values converge onto clusters, so a node may coincide with an eigenvalue; the
// candidates are therefore midpoints beside theta_j*, between it and the nearest nodes below
// and above that differ from it by more than 1e-8 of the nodes' scale (a, predicted fraction
// at or below: c_a; b, predicted c_{b-1}).
// out[0] = the candidate whose prediction is nearer 1/2 among those strictly inside (0, 1),
// out[1] = its prediction, or -1 when there is none (or T is not finite).
__global__ void quadrature_median_kernel(const LanczosState* stt, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  out[0] = 0.0;
  out[1] = -1.0;
  double d[kMaxT], z[kMaxT];
  int m = 0;
  if (!gauss_rule_thread(stt, d, z, &m)) return;
  // cumulative weights; js = the first node at which they reach 1/2
  double cw[kMaxT];
  double acc = 0.0;
  int js = -1;
  for (int i = 0; i < m; ++i) {
    acc += z[i];
    cw[i] = acc;
    if (js < 0 && acc >= 0.5) js = i;
  }
  if (js < 0) js = m - 1;
  // Two nodes may sit on one cluster, and their midpoint is then the clustered eigenvalue:
  // the neighbours taken are the nearest nodes that differ from theta_js by more than sep.
  const double sep = 1e-8 * fmax(fmax(d[m - 1] - d[0], fmax(fabs(d[0]), fabs(d[m - 1]))), 1e-300);
  int lo_i = js - 1;
  while (lo_i >= 0 && d[js] - d[lo_i] <= sep) --lo_i;
  int hi_i = js + 1;
  while (hi_i < m && d[hi_i] - d[js] <= sep) ++hi_i;
  const double lo_cut = 1e-12, hi_cut = 1.0 - 1e-12;
  double best = 0.0, best_pred = -1.0;
  if (lo_i >= 0 && cw[lo_i] > lo_cut && cw[lo_i] < hi_cut) {
    best = 0.5 * (d[lo_i] + d[js]);
    best_pred = cw[lo_i];
  }
  if (hi_i < m) {
    const double pu = cw[hi_i - 1];   // every node up to hi_i - 1 lies at or below the midpoint
    if (pu > lo_cut && pu < hi_cut && (best_pred < 0.0 || fabs(pu - 0.5) < fabs(best_pred - 0.5))) {
      best = 0.5 * (d[js] + d[hi_i]);
      best_pred = pu;
    }
  }
  if (best_pred < 0.0 || !isfinite(best)) return;
  out[0] = best;
  out[1] = best_pred;
}

// Count-to-threshold by stochastic Lanczos quadrature (Ubaru, Chen and Saad 2017).  State v
// holds the Lanczos tridiagonal of A from probe v; the nodes of A' = eps A are eps times its
// nodes.  By the Chebyshev-Markov-Stieltjes inequalities, at any x the probe's spectral
// distribution F_v(x) is at least L_v(x) = w_0 + ... + w_{j-2}, theta_{j-1} being the last
// node <= x.  out[0] = the smallest node x of all probes with
// n (mean_v L_v(x) - z stderr) >= k, out[1] = 1; out[1] = 0 when no node qualifies or a
// rule failed.  Threads 0 .. probes-1 build the rules, then every thread scans candidates.
constexpr int kSlqMaxProbes = 16;

__global__ void __launch_bounds__(256) slq_threshold_kernel(const LanczosState* states, int probes, double eps,
                                                            double n, double k, double z, double* out) {
  __shared__ double nodes[kSlqMaxProbes][kMaxT];
  __shared__ double cum[kSlqMaxProbes][kMaxT];   // cum[v][i] = w_0 + ... + w_i
  __shared__ int msz[kSlqMaxProbes];
  __shared__ int ok_all;
  __shared__ double red[256];
  const int tid = threadIdx.x;
  if (tid == 0) ok_all = 1;
  __syncthreads();
  if (tid < probes) {
    double d[kMaxT], w[kMaxT];
    int m = 0;
    if (!gauss_rule_thread(states + tid, d, w, &m)) {
      atomicAnd(&ok_all, 0);
      m = 0;
    }
    double acc = 0.0;
    for (int i = 0; i < m; ++i) {
      const int src = eps > 0.0 ? i : m - 1 - i;   // eps < 0 reverses the order
      nodes[tid][i] = eps * d[src];
      acc += w[src];
      cum[tid][i] = acc;
    }
    msz[tid] = m;
  }
  __syncthreads();
  double best = INFINITY;
  if (ok_all) {
    for (int c = tid; c < probes * kMaxT; c += blockDim.x) {
      const int v = c / kMaxT, i = c % kMaxT;
      if (i >= msz[v]) continue;
      const double x = nodes[v][i];
      double L[kSlqMaxProbes];
      double mean = 0.0;
      for (int u = 0; u < probes; ++u) {
        int j = 0;
        while (j < msz[u] && nodes[u][j] <= x) ++j;   // nodes of probe u at or below x
        L[u] = j >= 2 ? cum[u][j - 2] : 0.0;
        mean += L[u];
      }
      mean /= probes;
      double ss = 0.0;
      for (int u = 0; u < probes; ++u) ss += (L[u] - mean) * (L[u] - mean);
      const double se = probes > 1 ? sqrt(ss / (probes - 1) / probes) : 0.0;
      if (n * (mean - z * se) >= k) best = fmin(best, x);
    }
  }
  red[tid] = best;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) red[tid] = fmin(red[tid], red[tid + s]);
    __syncthreads();
  }
  if (tid == 0) {
    out[0] = red[0];
    out[1] = isfinite(red[0]) ? 1.0 : 0.0;
  }
}

}  // namespace

qdwhp_status gemv_t(cudaStream_t st, int64_t m, int64_t n, const double* A, int64_t lda, const double* x, double* y) {
  if (n <= 0) return QDWHP_OK;
  const int warps_per_block = 8;
  gemv_t_kernel<<<ceil_div(n, warps_per_block), 32 * warps_per_block, 0, st>>>((int)m, (int)n, A, lda, x, y);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

size_t gemv_n_part_elems(int64_t m, int64_t n) { return (size_t)m * ceil_div(std::max<int64_t>(n, 1), kGemvChunk); }

qdwhp_status gemv_n(cudaStream_t st, int64_t m, int64_t n, const double* A, int64_t lda, const double* x, double* y,
                    double* part) {
  if (m <= 0) return QDWHP_OK;
  const int nchunks = ceil_div(std::max<int64_t>(n, 1), kGemvChunk);
  dim3 grid(ceil_div(m, 256), nchunks);
  gemv_n_part_kernel<<<grid, 256, 0, st>>>((int)m, (int)n, A, lda, x, part);
  QDWHP_LAUNCH_CHECK();
  sum_chunks_kernel<<<ceil_div(m, 256), 256, 0, st>>>((int)m, nchunks, part, y);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status fill_gaussian(cudaStream_t st, int64_t rows, int64_t cols, uint64_t seed, double scale, double* out,
                           int64_t ld) {
  const size_t count = (size_t)rows * cols;
  if (count == 0) return QDWHP_OK;
  fill_gaussian_kernel<<<grid1d(count, 256), 256, 0, st>>>(count, seed, scale, out, rows, ld);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status fill_uniform(cudaStream_t st, int64_t rows, int64_t cols, uint64_t seed, double* out, int64_t ld) {
  const size_t count = (size_t)rows * cols;
  if (count == 0) return QDWHP_OK;
  fill_uniform_kernel<<<grid1d(count, 256), 256, 0, st>>>(count, seed, out, rows, ld);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

size_t lanczos_ws_elems(int64_t m, int64_t n, int steps) {
  // Q (n x steps), w (n), y (m), h0/h1 (steps), gemv partials
  return (size_t)n * steps + n + m + 2 * (size_t)steps + gemv_n_part_elems(m, n) + 64;
}

qdwhp_status lanczos(cudaStream_t st, bool normal, int64_t m, int64_t n, const double* A, int64_t lda, int steps,
                     uint64_t seed, double* ws, LanczosState* stt) {
  steps = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)steps, n, (int64_t)kMaxT}));
  double* Q = ws;
  double* w = Q + (size_t)n * steps;
  double* y = w + n;
  double* h0 = y + m;
  double* h1 = h0 + steps;
  double* part = h1 + steps;
  QDWHP_CUDA_TRY(cudaMemsetAsync(stt, 0, sizeof(LanczosState), st));
  QDWHP_TRY(fill_uniform(st, n, 1, seed ^ kStreamLanczos, Q, n));
  normalize_kernel<<<1, 1024, 0, st>>>((int)n, Q);
  QDWHP_LAUNCH_CHECK();
  const int rows_blocks = ceil_div(n, 256);
  for (int j = 0; j < steps; ++j) {
    const double* qj = Q + (size_t)j * n;
    if (normal) {
      QDWHP_TRY(gemv_n(st, m, n, A, lda, qj, y, part));   // y = A q
      QDWHP_TRY(gemv_t(st, m, n, A, lda, y, w));          // w = A^T y
    } else {
      QDWHP_TRY(gemv_t(st, n, n, A, lda, qj, w));         // symmetric: A q = A^T q
    }
    dots_t_kernel<<<j + 1, 256, 0, st>>>((int)n, Q, n, w, h0);
    QDWHP_LAUNCH_CHECK();
    sub_qh_kernel<<<rows_blocks, 256, 0, st>>>((int)n, j + 1, Q, n, h0, w);
    QDWHP_LAUNCH_CHECK();
    dots_t_kernel<<<j + 1, 256, 0, st>>>((int)n, Q, n, w, h1);
    QDWHP_LAUNCH_CHECK();
    sub_qh_kernel<<<rows_blocks, 256, 0, st>>>((int)n, j + 1, Q, n, h1, w);
    QDWHP_LAUNCH_CHECK();
    lanczos_finish_kernel<<<1, 1024, 0, st>>>((int)n, j, steps, h0, w, Q + (size_t)(j + 1) * n * (j + 1 < steps),
                                               stt);
    QDWHP_LAUNCH_CHECK();
  }
  tridiag_extremes_kernel<<<1, 32, 0, st>>>(stt);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status slq_threshold(cudaStream_t st, const LanczosState* states, int probes, double eps, int64_t n, int64_t k,
                           double z, double* out_dev) {
  if (probes < 1 || probes > kSlqMaxProbes) return QDWHP_ERR_ARG;
  slq_threshold_kernel<<<1, 256, 0, st>>>(states, probes, eps, (double)n, (double)k, z, out_dev);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status quadrature_median(cudaStream_t st, const LanczosState* stt, double* out_dev) {
  quadrature_median_kernel<<<1, 32, 0, st>>>(stt, out_dev);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

}  // namespace qdwhp
