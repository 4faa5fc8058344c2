// FP64 GEMM on the GB300 FP64 tensor path (mma.sync m8n8k4 .f64, "DMMA").
//
// tcgen05 has no f64 kind, so FP64 contractions run on DMMA.  Measured on this
// part, DMMA peaks at ~1.05 TFLOP/s (DFMA ~1.01): one SM does only a few FP64
// flops per clock, so the kernel needs no deep pipelining to stay compute bound
// (a 64x64x16 tile step is ~36k clocks of DMMA work against ~1k clocks of load
// latency).  What matters is covering all 152 SMs and keeping many CTAs resident:
// 32x32 tiles everywhere, and split-K for outputs with few tiles.  Split-K writes per-slice partial sums that a second kernel adds
// in a fixed order, so results do not depend on scheduling.
#include "internal.h"

namespace qdwhp {

namespace {

constexpr int kBK = 16;
constexpr int kChunk = 64;      // K slice summed separately before joining the accumulator
constexpr int kGroupM = 16;     // tile rows per raster group
constexpr int kThreads = 128;   // 2 x 2 warps

__device__ __forceinline__ void dmma884(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

template <int BM, int BN, bool TA, bool TB>
__global__ void __launch_bounds__(kThreads) dgemm_kernel(int M, int N, int K, int kchunk, double alpha,
                                                         const double* A, int64_t lda, const double* B,
                                                         int64_t ldb, double beta, double* C, int64_t ldc,
                                                         int uplo, double diag_add, double* partial) {
  constexpr int WM = BM / 2, WN = BN / 2;
  constexpr int MT = WM / 8, NT = WN / 8;
  constexpr int A_LD = BM * kBK / kThreads, B_LD = BN * kBK / kThreads;
  // Row strides of 8 mod 16 doubles keep a warp's fragment reads at two wavefronts.
  __shared__ double As[kBK][BM + 8];
  __shared__ double Bs[kBK][BN + 8];

  // Grouped raster order over a 1-D grid: consecutive CTAs walk down kGroupM tile rows
  // before moving one tile column right, so the CTAs resident at any time touch a
  // narrow band of A and B that stays in L2 (row-major order re-streams all of A for
  // every tile column once A exceeds L2).
  const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  const int pid = blockIdx.x;
  const int group = pid / (kGroupM * tiles_n);
  const int first_m = group * kGroupM;
  const int gsize = min(tiles_m - first_m, kGroupM);
  const int tm = first_m + (pid % (kGroupM * tiles_n)) % gsize;
  const int tn = (pid % (kGroupM * tiles_n)) / gsize;
  const int m0 = tm * BM, n0 = tn * BN;
  if (uplo == LOWER && m0 + BM <= n0) return;   // tile strictly above the diagonal
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int g = lane >> 2, t4 = lane & 3;

  // Two-level accumulation: each kChunk-wide slice of K is summed into `part`, which is then
  // added to `acc`, so the rounding chain per output is K / kChunk + kChunk / 4 long instead
  // of K / 4 (the dot products here run over up to tens of thousands of terms).
  double acc[MT][NT][2], part[MT][NT][2];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[i][j][0] = acc[i][j][1] = part[i][j][0] = part[i][j][1] = 0.0;

  double ra[A_LD], rb[B_LD];
  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < A_LD; ++r) {
      const int e = tid + kThreads * r;
      const int i = TA ? e / kBK : e % BM;
      const int kk = TA ? e % kBK : e / BM;
      const int gi = m0 + i, gk = k0 + kk;
      double v = 0.0;
      if (gi < M && gk < kend) v = TA ? A[gk + (int64_t)gi * lda] : A[gi + (int64_t)gk * lda];
      ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < B_LD; ++r) {
      const int e = tid + kThreads * r;
      const int j = TB ? e % BN : e / kBK;
      const int kk = TB ? e / BN : e % kBK;
      const int gj = n0 + j, gk = k0 + kk;
      double v = 0.0;
      if (gj < N && gk < kend) v = TB ? B[gj + (int64_t)gk * ldb] : B[gk + (int64_t)gj * ldb];
      rb[r] = v;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int r = 0; r < A_LD; ++r) {
      const int e = tid + kThreads * r;
      const int i = TA ? e / kBK : e % BM;
      const int kk = TA ? e % kBK : e / BM;
      As[kk][i] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < B_LD; ++r) {
      const int e = tid + kThreads * r;
      const int j = TB ? e % BN : e / kBK;
      const int kk = TB ? e / BN : e % kBK;
      Bs[kk][j] = rb[r];
    }
  };

  if (kbeg < kend) load(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += kBK) {
    __syncthreads();
    store();
    __syncthreads();
    if (k0 + kBK < kend) load(k0 + kBK);
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 4) {
      double af[MT], bf[NT];
#pragma unroll
      for (int i = 0; i < MT; ++i) af[i] = As[kk + t4][wm * WM + i * 8 + g];
#pragma unroll
      for (int j = 0; j < NT; ++j) bf[j] = Bs[kk + t4][wn * WN + j * 8 + g];
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j) dmma884(part[i][j], af[i], bf[j]);
    }
    if (((k0 - kbeg) / kBK) % (kChunk / kBK) == kChunk / kBK - 1 || k0 + kBK >= kend) {
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          acc[i][j][0] += part[i][j][0];
          acc[i][j][1] += part[i][j][1];
          part[i][j][0] = part[i][j][1] = 0.0;
        }
    }
  }

#pragma unroll
  for (int i = 0; i < MT; ++i) {
#pragma unroll
    for (int j = 0; j < NT; ++j) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int row = m0 + wm * WM + i * 8 + g;
        const int col = n0 + wn * WN + j * 8 + 2 * t4 + e;
        if (row >= M || col >= N) continue;
        if (uplo == LOWER && row < col) continue;
        if (partial != nullptr) {
          partial[(size_t)blockIdx.z * M * N + row + (size_t)col * M] = acc[i][j][e];
        } else {
          double v = alpha * acc[i][j][e];
          double* cp = C + row + (int64_t)col * ldc;
          if (beta != 0.0) v += beta * (*cp);
          if (row == col) v += diag_add;
          *cp = v;
        }
      }
    }
  }
}

__global__ void splitk_reduce_kernel(int M, int N, int splits, const double* partial, double alpha,
                                     double beta, double* C, int64_t ldc, int uplo, double diag_add) {
  const size_t total = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e % M), col = (int)(e / M);
    if (uplo == LOWER && row < col) continue;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += partial[(size_t)z * total + e];
    double v = alpha * s;
    double* cp = C + row + (int64_t)col * ldc;
    if (beta != 0.0) v += beta * (*cp);
    if (row == col) v += diag_add;
    *cp = v;
  }
}

template <int BM, int BN>
void launch(cudaStream_t st, bool ta, bool tb, dim3 grid, int M, int N, int K, int kchunk, double alpha,
            const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
            int uplo, double diag_add, double* partial) {
  if (!ta && !tb)
    dgemm_kernel<BM, BN, false, false><<<grid, kThreads, 0, st>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C,
                                                                ldc, uplo, diag_add, partial);
  else if (!ta && tb)
    dgemm_kernel<BM, BN, false, true><<<grid, kThreads, 0, st>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C,
                                                               ldc, uplo, diag_add, partial);
  else if (ta && !tb)
    dgemm_kernel<BM, BN, true, false><<<grid, kThreads, 0, st>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C,
                                                               ldc, uplo, diag_add, partial);
  else
    dgemm_kernel<BM, BN, true, true><<<grid, kThreads, 0, st>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C,
                                                              ldc, uplo, diag_add, partial);
}

constexpr int kMaxSplit = 16;
constexpr size_t kSplitMaxElems = size_t(1) << 22;   // split-K only for outputs up to 4M entries

}  // namespace

size_t gemm_splitk_ws_elems(int64_t m, int64_t n) {
  size_t mn = (size_t)m * (size_t)n;
  if (mn > kSplitMaxElems) return 0;
  return mn * kMaxSplit;
}

thread_local void* t_emu_ws = nullptr;
thread_local size_t t_emu_bytes = 0;

EmulationScope::EmulationScope(void* ws, size_t bytes) : prev_ws(t_emu_ws), prev_bytes(t_emu_bytes) {
  t_emu_ws = ws;
  t_emu_bytes = bytes;
}
EmulationScope::~EmulationScope() {
  t_emu_ws = prev_ws;
  t_emu_bytes = prev_bytes;
}

qdwhp_status gemm(cudaStream_t st, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                  int64_t ldc, Uplo uplo, double diag_add, double* splitk_ws, size_t splitk_ws_elems) {
  if (m < 0 || n < 0 || k < 0) return QDWHP_ERR_ARG;
  if (m == 0 || n == 0) return QDWHP_OK;
  if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || k > INT32_MAX / 2) return QDWHP_ERR_ARG;
  if (t_emu_ws != nullptr && m >= 128 && n >= 128 && k >= 256 && gemm_ozaki_ws_bytes(m, n, k) <= t_emu_bytes)
    return gemm_ozaki(st, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, uplo, diag_add, t_emu_ws,
                      t_emu_bytes);
  const int M = (int)m, N = (int)n, K = (int)k;
  // 32 x 32 tiles throughout: the DMMA pipe is slow enough that a small tile (96 registers,
  // many resident CTAs per SM) beats larger tiles (1.07 vs 1.00-1.02 TFLOP/s at 4096^3).
  constexpr int BM = 32, BN = 32;
  const int64_t tiles = (int64_t)ceil_div(M, BM) * ceil_div(N, BN) / (uplo == LOWER ? 2 : 1);
  int split = 1;
  const size_t mn = (size_t)M * N;
  if (splitk_ws != nullptr && tiles < kNumSMs && K >= 512 && mn <= kSplitMaxElems) {
    const int64_t target = (int64_t)tune_value(kTuneSplitkPerSM, std::max(M, N)) * kNumSMs;
    split = (int)std::min<int64_t>((target + tiles - 1) / std::max<int64_t>(tiles, 1), K / 256);
    split = std::min(split, kMaxSplit);
    while (split > 1 && (size_t)split * mn > splitk_ws_elems) --split;
    if (split < 1) split = 1;
  }
  int kchunk = (K + split - 1) / split;
  kchunk = ((kchunk + kBK - 1) / kBK) * kBK;
  if (split > 1) split = (K + kchunk - 1) / kchunk;
  dim3 grid(ceil_div(M, BM) * ceil_div(N, BN), 1, split);
  double* partial = split > 1 ? splitk_ws : nullptr;
  // algorithmic flops: 2 m n k, or n (n + 1) k for the lower triangle only
  const double flops = (uplo == LOWER) ? (double)N * (N + 1) * K : 2.0 * M * N * K;
  int prof_slot = -1;
  if (gemm_prof_enabled()) {
    const double shape[5] = {(double)M, (double)N, (double)K, (double)(uplo == LOWER), (double)split};
    prof_slot = gemm_prof_start(st, flops, shape);
  }
  launch<BM, BN>(st, ta, tb, grid, M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, uplo, diag_add, partial);
  QDWHP_LAUNCH_CHECK();
  if (split > 1) {
    const int blocks = (int)std::min<size_t>((mn + 255) / 256, 4 * kNumSMs);
    splitk_reduce_kernel<<<blocks, 256, 0, st>>>(M, N, split, partial, alpha, beta, C, ldc, uplo, diag_add);
    QDWHP_LAUNCH_CHECK();
  }
  if (prof_slot >= 0) gemm_prof_stop(st, prof_slot);
  return QDWHP_OK;
}

namespace {

// FP32 GEMM on the CUDA cores (FFMA), for the reduced-precision QDWH steps.  64 x 64 CTA
// tiles, 256 threads, 4 x 4 outputs per thread in a strided layout (rows ty + 16 i,
// columns tx + 16 j) so that the shared-memory reads of a warp are broadcasts.
constexpr int kSBK = 16;
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, float alpha, const float* A, int64_t lda,
                                                    const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                                                    int uplo, float diag_add) {
  constexpr int BM = 64, BN = 64;
  __shared__ float As[kSBK][BM + 4];
  __shared__ float Bs[kSBK][BN + 4];
  const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  const int pid = blockIdx.x;
  const int group = pid / (kGroupM * tiles_n);
  const int first_m = group * kGroupM;
  const int gsize = min(tiles_m - first_m, kGroupM);
  const int tm = first_m + (pid % (kGroupM * tiles_n)) % gsize;
  const int tn = (pid % (kGroupM * tiles_n)) / gsize;
  const int m0 = tm * BM, n0 = tn * BN;
  if (uplo == LOWER && m0 + BM <= n0) return;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  float ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + 256 * r;
      const int i = TA ? e / kSBK : e % BM;
      const int kk = TA ? e % kSBK : e / BM;
      const int gi = m0 + i, gk = k0 + kk;
      float v = 0.f;
      if (gi < M && gk < K) v = TA ? A[gk + (int64_t)gi * lda] : A[gi + (int64_t)gk * lda];
      ra[r] = v;
      const int j = TB ? e % BN : e / kSBK;
      const int kb = TB ? e / BN : e % kSBK;
      const int gj = n0 + j, gkb = k0 + kb;
      float w = 0.f;
      if (gj < N && gkb < K) w = TB ? B[gj + (int64_t)gkb * ldb] : B[gkb + (int64_t)gj * ldb];
      rb[r] = w;
    }
  };
  if (K > 0) load(0);
  for (int k0 = 0; k0 < K; k0 += kSBK) {
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + 256 * r;
      As[TA ? e % kSBK : e / BM][TA ? e / kSBK : e % BM] = ra[r];
      Bs[TB ? e / BN : e % kSBK][TB ? e % BN : e / kSBK] = rb[r];
    }
    __syncthreads();
    if (k0 + kSBK < K) load(k0 + kSBK);
#pragma unroll
    for (int kk = 0; kk < kSBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = m0 + ty + 16 * i, col = n0 + tx + 16 * j;
      if (row >= M || col >= N) continue;
      if (uplo == LOWER && row < col) continue;
      float v = alpha * acc[i][j];
      float* cp = C + row + (int64_t)col * ldc;
      if (beta != 0.f) v += beta * (*cp);
      if (row == col) v += diag_add;
      *cp = v;
    }
}

}  // namespace

thread_local void* t_f32tc_ws = nullptr;
thread_local size_t t_f32tc_bytes = 0;

Fp32TensorScope::Fp32TensorScope(void* ws, size_t bytes) : prev_ws(t_f32tc_ws), prev_bytes(t_f32tc_bytes) {
  t_f32tc_ws = ws;
  t_f32tc_bytes = bytes;
}
Fp32TensorScope::~Fp32TensorScope() {
  t_f32tc_ws = prev_ws;
  t_f32tc_bytes = prev_bytes;
}

qdwhp_status gemm(cudaStream_t st, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha, const float* A,
                  int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc, Uplo uplo,
                  float diag_add) {
  if (m < 0 || n < 0 || k < 0) return QDWHP_ERR_ARG;
  if (m == 0 || n == 0) return QDWHP_OK;
  if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || k > INT32_MAX / 2) return QDWHP_ERR_ARG;
  // Below 256 the slice splitting and the 128 x 128 tiles cost more than the CUDA-core kernel
  // (products of the triangular-solve recursion ran at 26 TFLOP/s FP32-equivalent at 128).
  if (t_f32tc_ws != nullptr && m >= 256 && n >= 256 && k >= 256 && gemm_bf16x6_ws_bytes(m, n, k) <= t_f32tc_bytes)
    return gemm_bf16x6(st, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, uplo, diag_add, t_f32tc_ws,
                       t_f32tc_bytes);
  const int M = (int)m, N = (int)n, K = (int)k;
  dim3 grid(ceil_div(M, 64) * ceil_div(N, 64));
  if (!ta && !tb)
    sgemm_kernel<false, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, uplo, diag_add);
  else if (!ta && tb)
    sgemm_kernel<false, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, uplo, diag_add);
  else if (ta && !tb)
    sgemm_kernel<true, false><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, uplo, diag_add);
  else
    sgemm_kernel<true, true><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, uplo, diag_add);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

}  // namespace qdwhp
