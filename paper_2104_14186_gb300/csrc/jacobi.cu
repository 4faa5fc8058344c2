// Reduced problems of the Rayleigh-Ritz step (Algorithm 1 step 6, Algorithm 2 step 6)
// by one-sided (Hestenes) Jacobi, plus selection, ordering and gathers.
//
// A sweep visits every column pair once in the round-robin ("circle method")
// order: nc - 1 rounds of nc / 2 disjoint pairs (a dummy column pads odd nc).  The
// pairs of a round are independent: a warp takes a pair, forms ||g_p||^2, ||g_q||^2
// and g_p^T g_q, and applies the plane rotation that makes the two columns
// orthogonal to G and to the accumulated Vj.  A whole sweep is one cooperative
// launch with a grid barrier between rounds.
//   - SVD: G = A Q2 (m x ell): sigma_i = ||w_i||, U = W Sigma^{-1}, V~ = Vj.
//   - EIG: G = M + sigma I with M = Q2^T A Q2 and sigma >= ||M||_2, so G is positive
//     semidefinite and its right singular vectors are eigenvectors of M; the
//     eigenvalues are then taken as Rayleigh quotients v_i^T M v_i.
#include <cooperative_groups.h>

#include <mutex>

#include "internal.h"
#include "krylov.h"

namespace cg = cooperative_groups;

namespace qdwhp {

namespace {

__device__ __forceinline__ void pair_of(int r, int h, int N, int& p, int& q) {
  if (h == 0) {
    p = N - 1;
    q = r;
  } else {
    p = (r + h) % (N - 1);
    q = (r - h + N - 1) % (N - 1);
  }
}

// Per-lane sums of one row: ||g_p||^2, ||g_q||^2 plainly, g_p^T g_q in double-double
// (TwoProduct, then TwoSum into (c, ce)).
__device__ __forceinline__ void accumulate_comp(double x, double y, double& a, double& b, double& c, double& ce) {
  a = fma(x, x, a);
  b = fma(y, y, b);
  const double pr = x * y;
  const double pe = fma(x, y, -pr);
  const double t = c + pr;
  const double z = t - c;
  ce += ((c - (t - z)) + (pr - z)) + pe;
  c = t;
}

// Warp sum of the double-double (c, ce) with TwoSum at every level; returns c + ce.
__device__ __forceinline__ double warp_sum_comp(double c, double ce) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double c2 = __shfl_xor_sync(0xffffffffu, c, o), e2 = __shfl_xor_sync(0xffffffffu, ce, o);
    const double t = c + c2;
    const double z = t - c;
    ce += e2 + ((c - (t - z)) + (c2 - z));
    c = t;
  }
  return c + ce;
}

// Lane 0 records the normalised inner product and, when it exceeds tol, forms the rotation
// that orthogonalises the pair; the decision and (cs, sn) are broadcast to the warp.
__device__ __forceinline__ int rotation_from_sums(double a, double b, double c, double tol, JacobiState* jst,
                                                  double& cs, double& sn) {
  const int lane = threadIdx.x & 31;
  int do_rot = 0;
  cs = 1.0;
  sn = 0.0;
  if (lane == 0) {
    if (!isfinite(a) || !isfinite(b) || !isfinite(c)) {
      atomicExch(&jst->nonfinite, 1);
    } else if (a > 0.0 && b > 0.0 && c != 0.0) {
      const double off = fabs(c) / sqrt(a * b);
      atomicMax(&jst->max_off_bits, (unsigned long long)__double_as_longlong(off));
      if (off > tol) {
        const double zeta = (b - a) / (2.0 * c);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        cs = 1.0 / sqrt(1.0 + t * t);
        sn = cs * t;
        do_rot = 1;
      }
    }
  }
  do_rot = __shfl_sync(0xffffffffu, do_rot, 0);
  cs = __shfl_sync(0xffffffffu, cs, 0);
  sn = __shfl_sync(0xffffffffu, sn, 0);
  return do_rot;
}

// Orthogonalise columns p and q of G (length mg) and rotate the same columns of Vj
// (length nc), by one warp: the lanes stride over the rows, the sums are combined with
// shuffles, lane 0 forms the rotation and broadcasts it.  ||g_p||^2 and ||g_q||^2 are
// summed plainly; g_p^T g_q, which decides convergence and goes to zero, is summed in
// double-double (TwoProduct and TwoSum) once the sweep is near convergence (comp != 0),
// so that it is accurate far below sqrt(mg) u and the stopping test can ask for
// orthogonality at the level of u.
__device__ void rotate_pair_warp(int p, int q, int mg, int nc, double* G, int64_t ldg, double* Vj, int64_t ldv,
                                 double tol, int comp, JacobiState* jst) {
  const int lane = threadIdx.x & 31;
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
  double* gp = G + (int64_t)p * ldg;
  double* gq = G + (int64_t)q * ldg;
  double a = 0.0, b = 0.0, c = 0.0, ce = 0.0;
  if (comp) {
    for (int i = lane; i < mg; i += 32) accumulate_comp(gp[i], gq[i], a, b, c, ce);
    c = warp_sum_comp(c, ce);
  } else {
    for (int i = lane; i < mg; i += 32) {
      const double x = gp[i], y = gq[i];
      a = fma(x, x, a);
      b = fma(y, y, b);
      c = fma(x, y, c);
    }
    c = warp_sum(c);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  double cs, sn;
  if (!rotation_from_sums(a, b, c, tol, jst, cs, sn)) return;
  for (int i = lane; i < mg; i += 32) {
    const double x = gp[i], y = gq[i];
    gp[i] = cs * x - sn * y;
    gq[i] = sn * x + cs * y;
  }
  double* vp = Vj + (int64_t)p * ldv;
  double* vq = Vj + (int64_t)q * ldv;
  for (int i = lane; i < nc; i += 32) {
    const double x = vp[i], y = vq[i];
    vp[i] = cs * x - sn * y;
    vq[i] = sn * x + cs * y;
  }
}

// The same pair update for columns of at most 32 R rows (mg, nc <= 32 R): the four columns
// are loaded into registers once, up front, so a pair costs one round trip to L2 instead of
// one per 32 rows; the arithmetic and its order are those of rotate_pair_warp.
template <int R>
__device__ void rotate_pair_warp_reg(int p, int q, int mg, int nc, double* G, int64_t ldg, double* Vj, int64_t ldv,
                                     double tol, int comp, JacobiState* jst) {
  const int lane = threadIdx.x & 31;
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
  double* gp = G + (int64_t)p * ldg;
  double* gq = G + (int64_t)q * ldg;
  double* vp = Vj + (int64_t)p * ldv;
  double* vq = Vj + (int64_t)q * ldv;
  double x[R], y[R], u[R], v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    x[r] = i < mg ? gp[i] : 0.0;
    y[r] = i < mg ? gq[i] : 0.0;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    u[r] = i < nc ? vp[i] : 0.0;
    v[r] = i < nc ? vq[i] : 0.0;
  }
  double a = 0.0, b = 0.0, c = 0.0, ce = 0.0;
  if (comp) {
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (lane + 32 * r < mg) accumulate_comp(x[r], y[r], a, b, c, ce);
    c = warp_sum_comp(c, ce);
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (lane + 32 * r < mg) {
        a = fma(x[r], x[r], a);
        b = fma(y[r], y[r], b);
        c = fma(x[r], y[r], c);
      }
    }
    c = warp_sum(c);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  double cs, sn;
  if (!rotation_from_sums(a, b, c, tol, jst, cs, sn)) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    if (i < mg) {
      gp[i] = cs * x[r] - sn * y[r];
      gq[i] = sn * x[r] + cs * y[r];
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane + 32 * r;
    if (i < nc) {
      vp[i] = cs * u[r] - sn * v[r];
      vq[i] = sn * u[r] + cs * v[r];
    }
  }
}

// One full sweep (N - 1 rounds) in one cooperative launch: every warp takes pairs of the
// round, and the grid meets at a barrier between rounds.
constexpr int kSweepMaxThreads = 512;   // up to 16 warps (pairs) per CTA, at most one CTA per SM
__global__ void __launch_bounds__(kSweepMaxThreads) jacobi_sweep_kernel(int mg, int nc, int N, double* G, int64_t ldg,
                                                                        double* Vj, int64_t ldv, double tol, int comp,
                                                                        JacobiState* jst) {
  cg::grid_group grid = cg::this_grid();
  const int wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nw = gridDim.x * wpb;
  for (int r = 0; r < N - 1; ++r) {
    for (int h = gw; h < N / 2; h += nw) {
      int p, q;
      pair_of(r, h, N, p, q);
      if (p < nc && q < nc) rotate_pair_warp(p, q, mg, nc, G, ldg, Vj, ldv, tol, comp, jst);
    }
    grid.sync();
  }
}

// Sweep kernel of the register-resident pair update (columns of at most 32 R rows).
constexpr int kSweepRegMaxThreads = 256;
template <int R>
__global__ void __launch_bounds__(kSweepRegMaxThreads) jacobi_sweep_reg_kernel(int mg, int nc, int N, double* G,
                                                                               int64_t ldg, double* Vj, int64_t ldv,
                                                                               double tol, int comp,
                                                                               JacobiState* jst) {
  cg::grid_group grid = cg::this_grid();
  const int wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nw = gridDim.x * wpb;
  for (int r = 0; r < N - 1; ++r) {
    for (int h = gw; h < N / 2; h += nw) {
      int p, q;
      pair_of(r, h, N, p, q);
      if (p < nc && q < nc) rotate_pair_warp_reg<R>(p, q, mg, nc, G, ldg, Vj, ldv, tol, comp, jst);
    }
    grid.sync();
  }
}

// Launch shape of a sweep: at most one CTA per SM (the budget of the cooperative-launch gate).
// A pair is one warp's work, and an SM's FP64 pipe is the bottleneck once it holds a few
// warps, so the pairs are first spread over the SMs at min_warps each (2 unless tuned); only
// when there are more pairs than that (long rounds) does a CTA take more warps, up to 16, to
// hide the latency of the column loads.
struct SweepShape {
  int grid;
  int threads;
};
SweepShape sweep_shape(int pairs, int max_threads, int min_warps) {
  static std::once_flag once;
  static int max_blocks = 0;
  std::call_once(once, [] {
    int dev = 0, sms = kNumSMs;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    max_blocks = sms;
  });
  const int max_warps = max_threads / 32;
  const int least = std::max(1, std::min(max_warps, min_warps));
  const int warps = std::max(least, std::min(max_warps, (pairs + max_blocks - 1) / max_blocks));
  const int grid = std::max(1, std::min(max_blocks, (pairs + warps - 1) / warps));
  return {grid, warps * 32};
}

__global__ void column_norms_kernel(int mg, const double* G, int64_t ldg, double* norms) {
  __shared__ double red[32];
  const double* g = G + (int64_t)blockIdx.x * ldg;
  double acc = 0.0;
  for (int i = threadIdx.x; i < mg; i += blockDim.x) acc += g[i] * g[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) norms[blockIdx.x] = sqrt(acc);
}

__global__ void column_dots_kernel(int mg, const double* V, int64_t ldv, const double* MV, int64_t ldmv, double* d) {
  __shared__ double red[32];
  const double* v = V + (int64_t)blockIdx.x * ldv;
  const double* w = MV + (int64_t)blockIdx.x * ldmv;
  double acc = 0.0;
  for (int i = threadIdx.x; i < mg; i += blockDim.x) acc += v[i] * w[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) d[blockIdx.x] = acc;
}

// Rank sort of the selected keys (one CTA; O(n^2) comparisons, n <= a few thousand).
__global__ void select_sort_kernel(int n, const double* vals, double sign, double thresh, int* order, int* count) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double ki = sign * vals[i];
    if (!(ki <= thresh)) continue;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double kj = sign * vals[j];
      if (!(kj <= thresh)) continue;
      if (kj < ki || (kj == ki && j < i)) ++rank;
    }
    order[rank] = i;
    atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *count = cnt;
}

__global__ void gather_columns_kernel(int rows, int k, const double* in, int64_t ldin, const int* order,
                                      const double* norms, double* out, int64_t ldout) {
  const size_t total = (size_t)rows * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), r = (int)(e / rows);
    const int src = order[r];
    double v = in[i + (int64_t)src * ldin];
    if (norms != nullptr) v /= norms[src];
    out[i + (int64_t)r * ldout] = v;
  }
}

__global__ void gather_values_kernel(int k, const double* vals, const int* order, double* out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < k) out[r] = vals[order[r]];
}

}  // namespace

qdwhp_status jacobi_onesided(cudaStream_t st, int64_t mg, int64_t nc, double* G, int64_t ldg, double* Vj, int64_t ldv,
                             int max_sweeps, double tol, JacobiState* jst_dev, JacobiState* jst_host, int* sweeps_out,
                             int* conv_out) {
  *sweeps_out = 0;
  *conv_out = 0;
  QDWHP_TRY(set_matrix(st, nc, nc, 0.0, 1.0, Vj, ldv));
  if (nc <= 1) {
    *conv_out = 1;
    return QDWHP_OK;
  }
  const int N = (int)(nc + (nc & 1));
  // columns of at most 512 rows stay in registers during a pair update
  const int64_t len = std::max(mg, nc);
  const void* fn = (const void*)jacobi_sweep_kernel;
  int max_threads = kSweepMaxThreads;
  if (len <= 128) {
    fn = (const void*)jacobi_sweep_reg_kernel<4>;
  } else if (len <= 256) {
    fn = (const void*)jacobi_sweep_reg_kernel<8>;
  } else if (len <= 512) {
    fn = (const void*)jacobi_sweep_reg_kernel<16>;
  }
  if (len <= 512) max_threads = kSweepRegMaxThreads;
  const SweepShape shape = sweep_shape(N / 2, max_threads, tune_value(kTuneJacobiWarps, nc));
  // Converged when the largest normalised inner product of a sweep is <= tol, or, once it
  // is below sqrt(mg) u (the level of a plain dot product's rounding), when a sweep no
  // longer reduces it by 4x: rotations of that size only stir rounding noise.
  const double floor_tol = std::max(tol, 2.220446049250313e-16 * std::sqrt((double)std::max<int64_t>(mg, 1)));
  double prev = INFINITY;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    QDWHP_CUDA_TRY(cudaMemsetAsync(jst_dev, 0, sizeof(JacobiState), st));
    int mg_i = (int)mg, nc_i = (int)nc, N_i = N;
    // compensated inner products only when they matter: a tight target, near convergence
    int comp = (tol < 1e-13 && prev < 1e-8) ? 1 : 0;
    void* args[] = {&mg_i, &nc_i, &N_i, &G, &ldg, &Vj, &ldv, &tol, &comp, &jst_dev};
    QDWHP_TRY(launch_cooperative(fn, dim3(shape.grid), dim3(shape.threads), args, 0, st));
    QDWHP_CUDA_TRY(cudaMemcpyAsync(jst_host, jst_dev, sizeof(JacobiState), cudaMemcpyDeviceToHost, st));
    QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
    *sweeps_out = sweep + 1;
    if (jst_host->nonfinite) return QDWHP_ERR_NONFINITE;
    double max_off;
    static_assert(sizeof(double) == sizeof(unsigned long long), "size");
    memcpy(&max_off, &jst_host->max_off_bits, sizeof(double));
    if (max_off <= tol || (max_off <= floor_tol && max_off > 0.25 * prev)) {
      *conv_out = 1;
      break;
    }
    prev = max_off;
  }
  return QDWHP_OK;
}

__global__ void normalize_columns_kernel(int rows, double* X, int64_t ldx, double* norms) {
  __shared__ double red[32];
  double* x = X + (int64_t)blockIdx.x * ldx;
  double acc = 0.0;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) acc += x[i] * x[i];
  acc = block_sum(acc, red);
  const double nrm = sqrt(acc);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) x[i] *= inv;
  if (norms != nullptr && threadIdx.x == 0) norms[blockIdx.x] = nrm;
}

qdwhp_status normalize_columns(cudaStream_t st, int64_t rows, int64_t ncols, double* X, int64_t ldx, double* norms) {
  if (ncols <= 0) return QDWHP_OK;
  normalize_columns_kernel<<<(int)ncols, 256, 0, st>>>((int)rows, X, ldx, norms);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status column_norms(cudaStream_t st, int64_t mg, int64_t nc, const double* G, int64_t ldg, double* norms) {
  if (nc <= 0) return QDWHP_OK;
  column_norms_kernel<<<(int)nc, 256, 0, st>>>((int)mg, G, ldg, norms);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status column_dots(cudaStream_t st, int64_t mg, int64_t nc, const double* V, int64_t ldv, const double* MV,
                         int64_t ldmv, double* d) {
  if (nc <= 0) return QDWHP_OK;
  column_dots_kernel<<<(int)nc, 256, 0, st>>>((int)mg, V, ldv, MV, ldmv, d);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status select_sort(cudaStream_t st, int64_t nvals, const double* vals, double sign, double thresh_key, int* order,
                         int* count_dev) {
  // Unselected tail entries stay 0, a valid index, so a later gather never reads out of range.
  QDWHP_CUDA_TRY(cudaMemsetAsync(order, 0, sizeof(int) * std::max<int64_t>(nvals, 1), st));
  select_sort_kernel<<<1, 1024, 0, st>>>((int)nvals, vals, sign, thresh_key, order, count_dev);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status gather_columns(cudaStream_t st, int64_t rows, int64_t k, const double* in, int64_t ldin, const int* order,
                            const double* inv_scale_by, double* out, int64_t ldout) {
  const size_t total = (size_t)rows * k;
  if (total == 0) return QDWHP_OK;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, 8 * kNumSMs));
  gather_columns_kernel<<<blocks, 256, 0, st>>>((int)rows, (int)k, in, ldin, order, inv_scale_by, out, ldout);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status gather_values(cudaStream_t st, int64_t k, const double* vals, const int* order, double* out) {
  if (k <= 0) return QDWHP_OK;
  gather_values_kernel<<<ceil_div(k, 256), 256, 0, st>>>((int)k, vals, order, out);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

}  // namespace qdwhp
