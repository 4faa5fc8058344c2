// Spectral bounds by Lanczos (Algorithm 1 step 1 "a few steps of the Lanczos
// iteration"; Algorithm 2 step 1 norm estimate on A^T A), HBM-bound GEMV kernels
// and the SplitMix64 start vectors.
//
// Lanczos runs with full reorthogonalisation (classical Gram-Schmidt, twice) and
// keeps every scalar on the device: the host only enqueues the steps.  The
// tridiagonal T (at most 64 x 64) is diagonalised by cyclic Jacobi in one warp;
// the extreme Ritz values and their residual norms beta_m |s_{m,i}| are the output.
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

// Cyclic Jacobi on the m x m tridiagonal T (one warp); writes the extreme Ritz values
// and residual norms beta_{m-1} |s_{m-1, i}|.
constexpr int kMaxT = 48;   // two 48 x 49 double arrays stay under the 48 KB static shared-memory limit
__global__ void tridiag_extremes_kernel(LanczosState* stt) {
  __shared__ double a[kMaxT][kMaxT + 1];
  __shared__ double v[kMaxT][kMaxT + 1];
  const int lane = threadIdx.x;
  const int m = max(1, min(stt->m, kMaxT));
  for (int e = lane; e < kMaxT * kMaxT; e += 32) {
    const int i = e % kMaxT, j = e / kMaxT;
    double t = 0.0;
    if (i < m && j < m) {
      if (i == j) t = stt->alpha[i];
      else if (i == j + 1) t = stt->beta[j];
      else if (j == i + 1) t = stt->beta[i];
    }
    a[i][j] = t;
    v[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncwarp();
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0;
    for (int e = lane; e < m * m; e += 32) {
      const int i = e % m, j = e / m;
      if (i < j) off += a[i][j] * a[i][j];
    }
    off = warp_sum(off);
    double fro = 0.0;
    for (int e = lane; e < m * m; e += 32) fro += a[e % m][e / m] * a[e % m][e / m];
    fro = warp_sum(fro);
    if (off <= 1e-36 * fro || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p) {
      for (int q = p + 1; q < m; ++q) {
        const double apq = a[p][q];
        if (apq == 0.0) continue;
        const double tau = (a[q][q] - a[p][p]) / (2.0 * apq);
        const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        __syncwarp();
        for (int i = lane; i < m; i += 32) {
          const double aip = a[i][p], aiq = a[i][q];
          a[i][p] = c * aip - s * aiq;
          a[i][q] = s * aip + c * aiq;
          const double vip = v[i][p], viq = v[i][q];
          v[i][p] = c * vip - s * viq;
          v[i][q] = s * vip + c * viq;
        }
        __syncwarp();
        for (int j = lane; j < m; j += 32) {
          const double apj = a[p][j], aqj = a[q][j];
          a[p][j] = c * apj - s * aqj;
          a[q][j] = s * apj + c * aqj;
        }
        __syncwarp();
        if (lane == 0) a[p][q] = a[q][p] = 0.0;
        __syncwarp();
      }
    }
  }
  if (lane == 0) {
    int imin = 0, imax = 0;
    for (int i = 1; i < m; ++i) {
      if (a[i][i] < a[imin][imin]) imin = i;
      if (a[i][i] > a[imax][imax]) imax = i;
    }
    const double bm = fabs(stt->beta[m - 1]);
    stt->out[0] = a[imin][imin];
    stt->out[1] = bm * fabs(v[m - 1][imin]);
    stt->out[2] = a[imax][imax];
    stt->out[3] = bm * fabs(v[m - 1][imax]);
  }
}

inline int grid1d(size_t total, int threads) {
  return (int)std::max<size_t>(1, std::min<size_t>((total + threads - 1) / threads, 16 * (size_t)kNumSMs));
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

}  // namespace qdwhp
