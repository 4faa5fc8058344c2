// FP32-accurate products on the BF16 tensor cores for the reduced-precision QDWH steps.
//
// Each FP32 entry x is split into three bfloat16 slices, x = h + m + l + d with
//     h = bf16(x),  m = bf16(x - h),  l = bf16(x - h - m)
// (every difference is exact in FP32, and each slice carries the next 8 significant bits, so
// |d| <= 2^-24 |x| up to the rounding of l).  The product of op(A) (M x K) and op(B) (K x N) is
// the sum of the six slice products with s + t <= 2,
//     hA hB + hA mB + mA hB + hA lB + mA mB + lA hB,
// the dropped ones (mA lB, lA mB, lA lB) being below 2^-25 |a| |b| per term.  All six
// accumulate in one FP32 tensor-memory accumulator, so the result carries FP32 rounding of the
// sums, like an FP32 GEMM: the "BF16x6" analogue of the 3xTF32 split (Henry, Tang, Heinecke,
// "Leveraging the bfloat16 artificial intelligence datatype for higher-precision computations",
// ARITH 2019).  Not part of the paper's method: it serves the FP32 Cholesky-based steps of
// QDWHP_MIXED.
//
// Kernel: one 128 x 128 output tile per CTA.  One thread of warp 4 feeds a 2-stage ring with
// TMA, a stage holding the three slices of op(A) and of op(B) for a 64-deep K block (6 x 16 KB),
// and issues that stage's 24 tcgen05.mma (6 slice pairs x 4 K steps of 16) as soon as it is
// full; each stage's MMAs commit to its "empty" mbarrier before the next block is copied in.
// The tensor core's own FP32 accumulation was measured to lose accuracy linearly with the
// number of accumulated MMAs (a 1540-MMA chain at K = 4100 left 25 times the error of an FP32
// product), so the partial sums are promoted: runs of two K blocks go to one of two 128-column
// tensor-memory buffers, and warps 0-3 add each finished run into FP32 registers (tcgen05.ld,
// round-to-nearest additions) while the next run fills the other buffer, then write
// C = alpha acc + beta C (+ diag_add on the diagonal).  Every wait is bounded; on a timeout the
// tile is written as NaN and err is set.
#include <cuda_bf16.h>

#include "internal.h"
#include "umma.cuh"

namespace qdwhp {

namespace {

constexpr int kB6Slices = 3;
constexpr int kB6Pairs = 6;
__constant__ unsigned char c_b6_s[kB6Pairs] = {0, 0, 1, 0, 1, 2};   // slice of op(A) per pair
__constant__ unsigned char c_b6_t[kB6Pairs] = {0, 1, 0, 2, 1, 0};   // slice of op(B) per pair
constexpr int kB6BM = 128, kB6BN = 128;
constexpr int kB6BK = umma::kAtomK;                                  // 64: one swizzle atom per slice
constexpr int kB6Stages = 2;
constexpr uint32_t kB6TileBytes = umma::kAtomBytes;                  // 16 KB: one slice, 128 rows x 64 K
constexpr uint32_t kB6OperandBytes = kB6Slices * kB6TileBytes;       // 48 KB
constexpr uint32_t kB6StageBytes = 2 * kB6OperandBytes;              // 96 KB
constexpr size_t kB6SmemBytes = (size_t)kB6Stages * kB6StageBytes + 1024;
constexpr int kB6Threads = 160;                                      // warps 0-3 flush, warp 4 copies + MMAs
constexpr int kB6RunBlocks = 2;   // K blocks (48 MMAs) accumulated in tensor memory before a flush

// Slices: out[s][r][l] (r < rows_pad, l < k_pad; zero outside rows x k) of src(r, l) =
// X[r + l ld] if rcontig else X[l + r ld].
__global__ void b6_split_kernel(int rows, int k, int rows_pad, int k_pad, const float* X, int64_t ld, int rcontig,
                                __nv_bfloat16* out) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int r0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
  __shared__ float tile[32][33];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = ty + 8 * q;
    int r, l;
    if (rcontig) { r = r0 + tx; l = l0 + a; } else { r = r0 + a; l = l0 + tx; }
    float v = 0.f;
    if (r < rows && l < k) v = rcontig ? X[r + (int64_t)l * ld] : X[l + (int64_t)r * ld];
    if (rcontig) tile[tx][a] = v; else tile[a][tx] = v;
  }
  __syncthreads();
  const size_t slice = (size_t)rows_pad * k_pad;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int rr = ty + 8 * q;
    const int r = r0 + rr, l = l0 + tx;
    if (r >= rows_pad || l >= k_pad) continue;
    const float x = tile[rr][tx];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r2);
    __nv_bfloat16* o = out + (size_t)r * k_pad + l;
    o[0] = h;
    o[slice] = m;
    o[2 * slice] = lo;
  }
}

__global__ void __launch_bounds__(kB6Threads, 1)
    b6_umma_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                   int k_pad, float alpha, float beta, float* C, int64_t ldc, int uplo, float diag_add, int* err) {
  extern __shared__ unsigned char b6_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)b6_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t bar_full[kB6Stages], bar_empty[kB6Stages];
  __shared__ __align__(8) uint64_t bar_run[2], bar_free[2], bar_done;
  __shared__ int s_abort, s_zero;
  const int m0 = blockIdx.y * kB6BM, n0 = blockIdx.x * kB6BN;
  if (uplo == LOWER && m0 + kB6BM <= n0) return;   // tile strictly above the diagonal
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nkb = k_pad / kB6BK;
  const int nruns = (nkb + kB6RunBlocks - 1) / kB6RunBlocks;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     umma::smem_addr(&tmem_base)),
                 "r"(2 * kB6BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 128) {
    for (int s = 0; s < kB6Stages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_addr(&bar_full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_addr(&bar_empty[s])));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_addr(&bar_run[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(umma::smem_addr(&bar_free[b])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_addr(&bar_done)));
    s_abort = 0;
    s_zero = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  volatile int* abort_flag = &s_abort;

  if (warp == 4) {
    if (lane == 0) {
      bool ok = true;
      const uint32_t sbase = umma::smem_addr(smem);
      auto issue_load = [&](int stage, int kb) {
        const uint32_t bar = umma::smem_addr(&bar_full[stage]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kB6StageBytes)
                     : "memory");
        const uint32_t dA = sbase + (uint32_t)stage * kB6StageBytes, dB = dA + kB6OperandBytes;
#pragma unroll
        for (int sl = 0; sl < kB6Slices; ++sl) {
          umma::tma_load_3d(dA + sl * kB6TileBytes, &mapA, kb * kB6BK, m0, sl, bar);
          umma::tma_load_3d(dB + sl * kB6TileBytes, &mapB, kb * kB6BK, n0, sl, bar);
        }
      };
      constexpr uint32_t idesc = umma::idesc_bf16_f32(kB6BM, kB6BN);
      // blocks [consumed, loaded) have a copy in flight whose "full" phase nobody has waited for
      int loaded = 0, consumed = 0;
      issue_load(0, 0);
      loaded = 1;
      for (int kb = 0; kb < nkb; ++kb) {
        const int stage = kb % kB6Stages;
        const int run = kb / kB6RunBlocks;
        const bool run_first = (kb % kB6RunBlocks) == 0;
        const bool run_last = (kb % kB6RunBlocks) == kB6RunBlocks - 1 || kb + 1 == nkb;
        // a run reuses the accumulator buffer of run - 2 once the flush warps have read it
        if (run_first && run >= 2 &&
            !umma::mbar_wait_or_abort(umma::smem_addr(&bar_free[run & 1]), (uint32_t)(((run >> 1) - 1) & 1),
                                      abort_flag)) {
          ok = false;
          break;
        }
        if (!umma::mbar_wait_or_abort(umma::smem_addr(&bar_full[stage]), (uint32_t)((kb / kB6Stages) & 1),
                                      abort_flag)) {
          ok = false;
          break;
        }
        consumed = kb + 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = sbase + (uint32_t)stage * kB6StageBytes, b0 = a0 + kB6OperandBytes;
        const uint32_t dcol = tmem + (uint32_t)((run & 1) * kB6BN);
#pragma unroll
        for (int p = 0; p < kB6Pairs; ++p) {
          const uint32_t as = a0 + (uint32_t)c_b6_s[p] * kB6TileBytes, bs = b0 + (uint32_t)c_b6_t[p] * kB6TileBytes;
#pragma unroll
          for (int kk = 0; kk < kB6BK / 16; ++kk) {
            const uint32_t accum = (run_first && p == 0 && kk == 0) ? 0u : 1u;
            umma::mma_bf16(dcol, umma::desc_sw128(as + 32 * kk), umma::desc_sw128(bs + 32 * kk), idesc, accum);
          }
        }
        umma::commit(umma::smem_addr(&bar_empty[stage]));
        if (run_last) umma::commit(umma::smem_addr(&bar_run[run & 1]));
        // Refill the other stage with block kb + 1 once the MMAs of block kb - 1 (its previous
        // contents) are done; block kb's MMAs, already queued, overlap that copy.
        if (kb + 1 < nkb) {
          const int other = (kb + 1) % kB6Stages;
          if (kb >= 1 && !umma::mbar_wait_or_abort(umma::smem_addr(&bar_empty[other]),
                                                   (uint32_t)(((kb - 1) / kB6Stages) & 1), abort_flag)) {
            ok = false;
            break;
          }
          issue_load(other, kb + 1);
          loaded = kb + 2;
        }
      }
      if (!ok) {
        *abort_flag = 1;
        // copies still in flight land before the CTA's shared memory is released (bounded)
        for (int b = consumed; b < loaded; ++b)
          umma::mbar_wait_or_abort(umma::smem_addr(&bar_full[b % kB6Stages]), (uint32_t)((b / kB6Stages) & 1),
                                   &s_zero);
      }
      umma::commit(umma::smem_addr(&bar_done));   // arrives when every MMA issued so far is complete
      // the tensor memory is freed below only after those MMAs are done (bounded)
      umma::mbar_wait_or_abort(umma::smem_addr(&bar_done), 0, &s_zero);
    }
    __syncwarp();
  } else {
    // Flush warps: each finished run (kB6RunBlocks K blocks) is added from tensor memory into
    // FP32 registers with round-to-nearest additions, so the long accumulation happens here
    // rather than inside the tensor core.  Thread = row m0 + 32 warp + lane, 128 columns.
    float acc[kB6BN];
#pragma unroll
    for (int j = 0; j < kB6BN; ++j) acc[j] = 0.f;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    bool good = true;
    for (int run = 0; run < nruns && good; ++run) {
      if (!umma::mbar_wait_or_abort(umma::smem_addr(&bar_run[run & 1]), (uint32_t)((run >> 1) & 1), abort_flag)) {
        good = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int h = 0; h < kB6BN / 32; ++h) {
        uint32_t v[32];
        umma::tmem_ld32(tmem + lane_base + (uint32_t)((run & 1) * kB6BN) + (uint32_t)(32 * h), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[32 * h + c] += __uint_as_float(v[c]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_addr(&bar_free[run & 1])) : "memory");
    }
    if (!good) *abort_flag = 1;
    if (!umma::mbar_wait_or_abort(umma::smem_addr(&bar_done), 0, abort_flag)) good = false;
    __syncwarp();
    good = good && !*abort_flag;
    const int i = m0 + warp * 32 + lane;
    if (i < M) {
#pragma unroll
      for (int c = 0; c < kB6BN; ++c) {
        const int j = n0 + c;
        if (j >= N || (uplo == LOWER && i < j)) continue;
        float x = good ? alpha * acc[c] : __int_as_float(0x7fc00000);
        float* cp = C + i + (int64_t)j * ldc;
        if (beta != 0.f) x = fmaf(beta, *cp, x);
        if (i == j) x += diag_add;
        *cp = x;
      }
    }
    if (!good && lane == 0) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kB6BN));
}

int round_up(int64_t a, int b) { return (int)(((a + b - 1) / b) * b); }

}  // namespace

size_t gemm_bf16x6_ws_bytes(int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  const size_t mp = round_up(m, kB6BM), np = round_up(n, kB6BN), kp = round_up(k, kB6BK);
  return (size_t)kB6Slices * (mp + np) * kp * 2 + 1024;
}

qdwhp_status gemm_bf16x6(cudaStream_t st, bool ta, bool tb, int64_t m, int64_t n, int64_t k, float alpha,
                         const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                         Uplo uplo, float diag_add, void* ws, size_t ws_bytes) {
  if (m < 0 || n < 0 || k < 0) return QDWHP_ERR_ARG;
  if (m == 0 || n == 0) return QDWHP_OK;
  if (m > (1 << 24) || n > (1 << 24) || k > (1 << 24)) return QDWHP_ERR_ARG;
  if (k == 0) return gemm(st, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, uplo, diag_add);
  if (ws == nullptr || ws_bytes < gemm_bf16x6_ws_bytes(m, n, k)) return QDWHP_ERR_NOMEM;
  static PerDeviceOnce attr;
  QDWHP_CUDA_TRY(attr.run(
      [] { return cudaFuncSetAttribute(b6_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kB6SmemBytes); }));
  const int mp = round_up(m, kB6BM), np = round_up(n, kB6BN), kp = round_up(k, kB6BK);
  __nv_bfloat16* Asl = (__nv_bfloat16*)ws;
  __nv_bfloat16* Bsl = Asl + (size_t)kB6Slices * mp * kp;
  int* err = (int*)(Bsl + (size_t)kB6Slices * np * kp);
  QDWHP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  // op(A) rows are contiguous iff A is not transposed; op(B) columns iff B is transposed
  b6_split_kernel<<<dim3(mp / 32, kp / 32), 256, 0, st>>>((int)m, (int)k, mp, kp, A, lda, ta ? 0 : 1, Asl);
  QDWHP_LAUNCH_CHECK();
  b6_split_kernel<<<dim3(np / 32, kp / 32), 256, 0, st>>>((int)n, (int)k, np, kp, B, ldb, tb ? 1 : 0, Bsl);
  QDWHP_LAUNCH_CHECK();
  CUtensorMap mapA, mapB;
  QDWHP_TRY(umma::slice_map(&mapA, (const unsigned short*)Asl, kB6Slices, mp, kp));
  QDWHP_TRY(umma::slice_map(&mapB, (const unsigned short*)Bsl, kB6Slices, np, kp));
  const double flops = (uplo == LOWER) ? (double)n * (n + 1) * k : 2.0 * m * n * k;
  int prof_slot = -1;
  if (gemm_prof_enabled()) {
    const double shape[5] = {(double)m, (double)n, (double)k, (double)(uplo == LOWER), -2.0};
    prof_slot = gemm_prof_start(st, flops, shape);
  }
  dim3 grid(np / kB6BN, mp / kB6BM);
  b6_umma_kernel<<<grid, kB6Threads, kB6SmemBytes, st>>>(mapA, mapB, (int)m, (int)n, kp, alpha, beta, C, ldc,
                                                          (int)uplo, diag_add, err);
  QDWHP_LAUNCH_CHECK();
  if (prof_slot >= 0) gemm_prof_stop(st, prof_slot);
  return QDWHP_OK;
}

}  // namespace qdwhp
