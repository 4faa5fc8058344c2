// FP64 GEMM emulated on the BF16 tensor cores by the Ozaki splitting scheme
// (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication and its applications", Numer. Algorithms
// 59 (2012); as run on low-precision tensor cores by Mukunoki, Ozaki, Ogita, Imamura, 2020).
// Not part of the paper's method: a faster route to FP64-accurate products on a part whose
// FP64 pipe is ~1/600 of its BF16 tensor rate.
//
// Each row i of op(A) is scaled by 2^-e_i (e_i: binary exponent of the row's largest
// magnitude, so every entry lies in (-1, 1)) and rounded to a 54-bit fixed-point integer,
// written in base 2^6 as 9 signed digits D_1..D_9 (|D| <= 63: exact in bfloat16).
// Columns of op(B) are split the same way with exponents f_j.  Then
//     C_ij = 2^(e_i + f_j) sum_{s,t} 2^(-6 (s + t)) (D^A_s D^B_t)_ij ,
// where every digit product D^A_s D^B_t is an exact integer matrix product: each term is
// < 2^12 in magnitude, so a sum over K <= 4096 terms stays below 2^24 and is exact in the
// FP32 accumulators of the tensor cores (bf16 x bf16 -> f32).  Each such product is scaled
// by its power of two and added into FP64 accumulators.  The pairs with s + t <= 12 are
// kept (60 of the 81).  The dropped pairs are a bias, not noise, where the digit products
// share a sign (a sum of squares): at most 6 K 63^2 2^-78 2^(e_i + f_j), below the K u
// 2^(e_i + f_j) rounding bound of an FP64 dot product of length K (one level fewer would put
// 64 times more bias on Gram diagonals).  Pairs
// of one level s + t share the scale 2^(-6 (s + t)), so they share an FP32 accumulator as
// long as it holds at most 4224 digit products (exact); it is flushed into FP64 when the
// level changes or the budget would be exceeded.
//
// Layout: digit slices are stored as [slice][row][k_pad] bfloat16 with K contiguous (op(A)
// rows, op(B) columns), zero-padded to 128-row, 128-deep blocks; the product kernel (TMA +
// tcgen05, below) streams a (slice pair, K block) sequence through a 3-stage ring in shared
// memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>

#include "internal.h"
#include "umma.cuh"

namespace qdwhp {

namespace {

constexpr int kOzS = 9;          // digits per entry
constexpr int kOzBeta = 6;       // bits per digit
constexpr int kOzT = 12;         // keep digit pairs with s + t <= kOzT (1-based)
constexpr int kOzBudget = 4224;  // FP32 exactness: at most this many digit products (each
                                 // < 2^12 in magnitude) in one accumulator: 4224 * 63^2 < 2^24
constexpr int kOzBM = 128, kOzBN = 128;   // row padding of the op(A) and op(B) digit slices
constexpr int kOzKPad = 128;              // K padding of the digit slices (one K block)
constexpr int kExpEmpty = -2000000000;   // no entry seen yet (row of zeros)
constexpr int kExpNonfinite = 1 << 20;   // a NaN or Inf in the row

struct PairTable {
  int npairs;
  unsigned char s[kOzS * kOzS];
  unsigned char t[kOzS * kOzS];
  unsigned char lev[kOzS * kOzS];
  double scale[kOzS * kOzS];
};
__constant__ PairTable c_pairs;

// ---- splitting ----

__global__ void oz_init_exp_kernel(int n, int* e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) e[i] = kExpEmpty;
}

// exps[r] = max over l of the binary exponent of |op(X)(r, l)| (frexp convention), or
// kExpNonfinite if the row holds a NaN/Inf.  src(r, l) = X[r + l ld] if rcontig else X[l + r ld].
__global__ void oz_exp_kernel(int rows, int k, const double* X, int64_t ld, int rcontig, int* exps) {
  // 32 x 32 tile, 256 threads: thread (tx, ty) reads 4 entries
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int r0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
  __shared__ int red[32][33];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = ty + 8 * q;   // the non-contiguous coordinate
    int r, l;
    if (rcontig) { r = r0 + tx; l = l0 + a; } else { r = r0 + a; l = l0 + tx; }
    int e = kExpEmpty;
    if (r < rows && l < k) {
      const double v = rcontig ? X[r + (int64_t)l * ld] : X[l + (int64_t)r * ld];
      if (!isfinite(v)) {
        e = kExpNonfinite;
      } else if (v != 0.0) {
        int ex;
        frexp(v, &ex);
        e = ex;
      }
    }
    // red[row within tile][col within tile]
    if (rcontig) red[tx][a] = e; else red[a][tx] = e;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    int m = kExpEmpty;
    for (int c = 0; c < 32; ++c) m = max(m, red[threadIdx.x][c]);
    const int r = r0 + threadIdx.x;
    if (r < rows && m != kExpEmpty) atomicMax(&exps[r], m);
  }
}

__device__ __forceinline__ unsigned short bf16_bits_of_small_int(int d) {
  // |d| <= 63: exactly representable; round-to-nearest conversion is exact
  const __nv_bfloat16 h = __int2bfloat16_rn(d);
  return *reinterpret_cast<const unsigned short*>(&h);
}

// Digit slices: out[s][r][l] (r < rows_pad, l < k_pad; zero outside rows x k).
__global__ void oz_split_kernel(int rows, int k, int rows_pad, int k_pad, const double* X, int64_t ld, int rcontig,
                                const int* exps, unsigned short* out) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int r0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
  __shared__ double tile[32][33];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = ty + 8 * q;
    int r, l;
    if (rcontig) { r = r0 + tx; l = l0 + a; } else { r = r0 + a; l = l0 + tx; }
    double v = 0.0;
    if (r < rows && l < k) v = rcontig ? X[r + (int64_t)l * ld] : X[l + (int64_t)r * ld];
    if (rcontig) tile[tx][a] = v; else tile[a][tx] = v;
  }
  __syncthreads();
  // write phase: thread (tx, ty) handles rows ty + 8 q, column tx (K contiguous)
  const size_t slice = (size_t)rows_pad * k_pad;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int rr = ty + 8 * q;
    const int r = r0 + rr, l = l0 + tx;
    if (r >= rows_pad || l >= k_pad) continue;
    const double v = tile[rr][tx];
    int e = (r < rows) ? exps[r] : kExpEmpty;
    long long X54 = 0;
    if (e != kExpEmpty && e != kExpNonfinite && v != 0.0) {
      // |v| 2^-e < 1; scaled by 2^54 it is exact, and rounding to an integer loses < 2^-55
      X54 = llrint(ldexp(v, 54 - e));
    }
    const unsigned long long U = (unsigned long long)(X54 < 0 ? -X54 : X54);
    const int sgn = X54 < 0 ? -1 : 1;
    unsigned short* o = out + (size_t)r * k_pad + l;
#pragma unroll
    for (int s = 0; s < kOzS; ++s) {
      const int d = (int)((U >> (kOzBeta * (kOzS - 1 - s))) & ((1u << kOzBeta) - 1));
      o[(size_t)s * slice] = bf16_bits_of_small_int(sgn * d);
    }
  }
}

// ---- the digit-product GEMM ----

// ---- tcgen05 (UMMA) digit-product kernel ----
//
// The 60 exact digit products run on the 5th-generation tensor cores as
// tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128, N = 128, K = 16).  Both operands are
// read from shared memory through matrix descriptors: K-major, 128-byte swizzle, i.e. 8-row
// atoms of 1024 bytes with 16-byte chunk c of row r stored at chunk c ^ (r % 8), which is the
// layout the TMA engine writes for a 64 x 128 box with the 128-byte swizzle.  The FP32 sums live
// in tensor memory (two 128-column accumulators), and every mbarrier wait is bounded: on a
// timeout the tile is written as NaN and err is set.
constexpr int kUmN = 128;
constexpr int kUmAtomK = umma::kAtomK;                           // K of one 128-byte swizzle atom row
constexpr int kUmBK = 128;                                      // K per stage: two atoms per operand
constexpr int kUmStages = 3;
constexpr uint32_t kUmAtomBytes = 128 * kUmAtomK * 2;           // 16 KB: 128 rows x 64 K
constexpr uint32_t kUmTileBytes = 128 * kUmBK * 2;              // 32 KB per operand and stage
constexpr uint32_t kUmStageBytes = 2 * kUmTileBytes;
constexpr size_t kUmSmemBytes = (size_t)kUmStages * kUmStageBytes + 1024;

// ---- warp-specialised TMA + tcgen05 digit-product kernel ----
//
// Warp 8 (one thread) feeds a 3-stage ring (128-deep K per stage) with TMA (cp.async.bulk.tensor, 128-byte swizzle
// written by the copy engine, each stage's "full" mbarrier counting the bytes) and issues the
// MMAs of a stage as soon as it is full; each stage's MMAs commit to its "empty" mbarrier, which
// releases the stage to the next copy.  A level run (digit pairs of one level, at most 4224
// digit products per accumulator) accumulates into one of two 128-column TMEM buffers and commits to that buffer's
// "run done" mbarrier.  Warps 0-7 only flush: for each run they wait on "run done", read the
// FP32 sums (tcgen05.ld), add them into their FP64 registers and arrive on the buffer's "free"
// mbarrier, which the issuing thread waits on before reusing the buffer two runs later.  The
// flush warps derive the run schedule from the pair table (no per-step synchronisation).
constexpr int kWsThreads = 288;
constexpr int kWsRunSteps = kOzBudget / kUmBK;   // K blocks per run at most (exact FP32 sums)

__global__ void __launch_bounds__(kWsThreads, 1)
    oz_umma_ws_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                      int k_pad, const int* __restrict__ ea, const int* __restrict__ eb, double alpha, double beta,
                      double* C, int64_t ldc, int uplo, double diag_add, int* err) {
  extern __shared__ unsigned char ws_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)ws_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t bar_full[kUmStages], bar_empty[kUmStages];
  __shared__ __align__(8) uint64_t bar_run[2], bar_free[2], bar_done;
  __shared__ int s_abort, s_zero;
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * kUmN;
  if (uplo == LOWER && m0 + 128 <= n0) return;   // tile strictly above the diagonal
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nkb = k_pad / kUmBK;
  const int npairs = c_pairs.npairs;
  const int total = npairs * nkb;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(umma::smem_addr(&tmem_base)),
                 "r"(2 * kUmN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 256) {
    for (int s = 0; s < kUmStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_addr(&bar_full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_addr(&bar_empty[s])));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_addr(&bar_run[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(umma::smem_addr(&bar_free[b])));
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
  bool ok = true;

  if (warp == 8) {
    if (lane == 0) {
      const uint32_t sbase = umma::smem_addr(smem);
      int lp = 0, lkb = 0;
      auto issue_load = [&](int stage) {
        const uint32_t bar = umma::smem_addr(&bar_full[stage]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kUmStageBytes)
                     : "memory");
        const uint32_t dA = sbase + (uint32_t)stage * kUmStageBytes, dB = dA + kUmTileBytes;
#pragma unroll
        for (int at = 0; at < kUmBK / kUmAtomK; ++at) {
          umma::tma_load_3d(dA + at * kUmAtomBytes, &mapA, lkb * kUmBK + at * kUmAtomK, m0, (int)c_pairs.s[lp], bar);
          umma::tma_load_3d(dB + at * kUmAtomBytes, &mapB, lkb * kUmBK + at * kUmAtomK, n0, (int)c_pairs.t[lp], bar);
        }
        if (++lkb == nkb) {
          lkb = 0;
          ++lp;
        }
      };
      // steps [consumed, loaded) have a copy in flight whose "full" phase nobody has waited for
      int loaded = 0, consumed = 0;
      for (int st = 0; st < kUmStages - 1 && st < total; ++st) {
        issue_load(st);
        loaded = st + 1;
      }
      const uint32_t idesc =
          (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kUmN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      int cp = 0, ckb = 0, steps_in_run = 0, run = 0;
      bool run_first = true;
      for (int step = 0; step < total && ok; ++step) {
        const int stage = step % kUmStages;
        if (!umma::mbar_wait_or_abort(umma::smem_addr(&bar_full[stage]), (uint32_t)((step / kUmStages) & 1), abort_flag)) {
          ok = false;
          break;
        }
        consumed = step + 1;
        if (run_first && run >= 2 &&
            !umma::mbar_wait_or_abort(umma::smem_addr(&bar_free[run & 1]), (uint32_t)(((run >> 1) - 1) & 1), abort_flag)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = sbase + (uint32_t)stage * kUmStageBytes, b0 = a0 + kUmTileBytes;
        const uint32_t dcol = tmem + (uint32_t)((run & 1) * kUmN);
#pragma unroll
        for (int kk = 0; kk < kUmBK / 16; ++kk) {
          // atom kk / 4, 32-byte K step kk % 4 inside it
          const uint32_t off = (uint32_t)(kk / 4) * kUmAtomBytes + (uint32_t)(kk % 4) * 32;
          const uint64_t da = umma::desc_sw128(a0 + off), db = umma::desc_sw128(b0 + off);
          const uint32_t accum = (run_first && kk == 0) ? 0u : 1u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
              "l"(da), "l"(db), "r"(idesc), "r"(accum));
        }
        umma::commit(umma::smem_addr(&bar_empty[stage]));
        ++steps_in_run;
        int np_ = cp, nkb_ = ckb + 1;
        if (nkb_ == nkb) {
          nkb_ = 0;
          ++np_;
        }
        const bool run_ends = np_ >= npairs || c_pairs.lev[np_] != c_pairs.lev[cp] || steps_in_run >= kWsRunSteps;
        if (run_ends) {
          umma::commit(umma::smem_addr(&bar_run[run & 1]));
          ++run;
          run_first = true;
          steps_in_run = 0;
        } else {
          run_first = false;
        }
        const int nxt = step + kUmStages - 1;
        if (nxt < total) {
          if (step >= 1 && !umma::mbar_wait_or_abort(umma::smem_addr(&bar_empty[(step - 1) % kUmStages]),
                                               (uint32_t)(((step - 1) / kUmStages) & 1), abort_flag)) {
            ok = false;
            break;
          }
          issue_load(nxt % kUmStages);
          loaded = nxt + 1;
        }
        cp = np_;
        ckb = nkb_;
      }
      if (!ok) {
        *abort_flag = 1;
        // copies still in flight land before the CTA's shared memory is released (bounded)
        for (int b = consumed; b < loaded; ++b)
          umma::mbar_wait_or_abort(umma::smem_addr(&bar_full[b % kUmStages]), (uint32_t)((b / kUmStages) & 1),
                                   &s_zero);
      }
      umma::commit(umma::smem_addr(&bar_done));   // every MMA issued so far
      // the tensor memory is freed below only after those MMAs are done (bounded)
      umma::mbar_wait_or_abort(umma::smem_addr(&bar_done), 0, &s_zero);
    }
    __syncwarp();
  } else {
    // flush warps: row (warp % 4) * 32 + lane, columns (warp / 4) * 64 + [0, 64)
    double acc64[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) acc64[j] = 0.0;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t col_base = (uint32_t)((warp >> 2) * 64);
    int run = 0;
    for (int p = 0; p < npairs && ok;) {
      int q = p;
      while (q < npairs && c_pairs.lev[q] == c_pairs.lev[p]) ++q;   // pairs [p, q) share a level
      const int level_steps = (q - p) * nkb;
      const double sc = c_pairs.scale[p];
      for (int done = 0; done < level_steps && ok; done += kWsRunSteps, ++run) {
        if (!umma::mbar_wait_or_abort(umma::smem_addr(&bar_run[run & 1]), (uint32_t)((run >> 1) & 1), abort_flag)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t v[32];
          umma::tmem_ld32(tmem + lane_base + (uint32_t)((run & 1) * kUmN) + col_base + (uint32_t)(32 * h), v);
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int j = 0; j < 32; ++j) acc64[32 * h + j] = fma((double)__uint_as_float(v[j]), sc, acc64[32 * h + j]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_addr(&bar_free[run & 1])) : "memory");
      }
      p = q;
    }
    if (!ok) *abort_flag = 1;
    if (!umma::mbar_wait_or_abort(umma::smem_addr(&bar_done), 0, abort_flag)) ok = false;
    // epilogue: C = alpha 2^(e_i + f_j) acc + beta C (+ diag_add on the diagonal)
    __syncwarp();
    const bool good = ok && !*abort_flag;
    const int i = m0 + (warp & 3) * 32 + lane;
    if (i < M) {
      const int e_i = ea[i];
#pragma unroll
      for (int c = 0; c < 64; ++c) {
        const int j = n0 + (int)col_base + c;
        if (j >= N || (uplo == LOWER && i < j)) continue;
        const int f_j = eb[j];
        double v;
        if (!good || e_i == kExpNonfinite || f_j == kExpNonfinite) {
          v = __longlong_as_double(0x7ff8000000000000ll);
        } else if (e_i == kExpEmpty || f_j == kExpEmpty) {
          v = 0.0;
        } else {
          v = alpha * ldexp(acc64[c], e_i + f_j);
        }
        double* cptr = C + i + (int64_t)j * ldc;
        if (beta != 0.0) v = fma(beta, *cptr, v);
        if (i == j) v += diag_add;
        *cptr = v;
      }
    }
    if (!good && lane == 0) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kUmN));
}

}  // namespace

namespace umma {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

}  // namespace

qdwhp_status slice_map(CUtensorMap* map, const unsigned short* base, int nslices, int rows_pad, int k_pad) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (enc == nullptr) {
    set_error_message("cuTensorMapEncodeTiled is not available from the driver");
    return QDWHP_ERR_CUDA;
  }
  const cuuint64_t dims[3] = {(cuuint64_t)k_pad, (cuuint64_t)rows_pad, (cuuint64_t)nslices};
  const cuuint64_t strides[2] = {(cuuint64_t)k_pad * 2, (cuuint64_t)rows_pad * k_pad * 2};
  const cuuint32_t box[3] = {(cuuint32_t)kAtomK, 128u, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error_message("cuTensorMapEncodeTiled rejected a bfloat16 slice tensor map");
    return QDWHP_ERR_CUDA;
  }
  return QDWHP_OK;
}

}  // namespace umma

namespace {

qdwhp_status launch_umma_ws(cudaStream_t st, int64_t m, int64_t n, int kp, int mp, int np, const unsigned short* Asl,
                            const unsigned short* Bsl, const int* ea, const int* eb, double alpha, double beta,
                            double* C, int64_t ldc, Uplo uplo, double diag_add, int* err) {
  static PerDeviceOnce attr;
  QDWHP_CUDA_TRY(attr.run([] {
    return cudaFuncSetAttribute(oz_umma_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUmSmemBytes);
  }));
  CUtensorMap mapA, mapB;
  QDWHP_TRY(umma::slice_map(&mapA, Asl, kOzS, mp, kp));
  QDWHP_TRY(umma::slice_map(&mapB, Bsl, kOzS, np, kp));
  dim3 grid(np / kUmN, mp / 128);
  oz_umma_ws_kernel<<<grid, kWsThreads, kUmSmemBytes, st>>>(mapA, mapB, (int)m, (int)n, kp, ea, eb, alpha, beta, C,
                                                            ldc, (int)uplo, diag_add, err);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

int ceil_to(int64_t a, int b) { return (int)(((a + b - 1) / b) * b); }

PerDeviceOnce g_pairs_once;

qdwhp_status upload_pairs() {
  const cudaError_t e = g_pairs_once.run([] {
    PairTable t;
    memset(&t, 0, sizeof(t));
    int p = 0;
    // most significant pairs first (any order is exact in FP32; FP64 adds in this order)
    for (int lev = 2; lev <= kOzT; ++lev)
      for (int s = 1; s <= kOzS; ++s) {
        const int tt = lev - s;
        if (tt < 1 || tt > kOzS) continue;
        t.s[p] = (unsigned char)(s - 1);
        t.t[p] = (unsigned char)(tt - 1);
        t.lev[p] = (unsigned char)lev;
        t.scale[p] = ldexp(1.0, -kOzBeta * lev);
        ++p;
      }
    t.npairs = p;
    return cudaMemcpyToSymbol(c_pairs, &t, sizeof(t));
  });
  if (e != cudaSuccess) {
    set_last_error(e, "upload of the digit-pair table", __FILE__, __LINE__);
    return QDWHP_ERR_CUDA;
  }
  return QDWHP_OK;
}

}  // namespace

size_t gemm_ozaki_ws_bytes(int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  const size_t mp = ceil_to(m, kOzBM), np = ceil_to(n, kOzBN), kp = ceil_to(k, kOzKPad);
  return (size_t)kOzS * (mp + np) * kp * 2 + (mp + np + 4) * sizeof(int) + 1024;
}

qdwhp_status gemm_ozaki(cudaStream_t st, bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                        const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                        int64_t ldc, Uplo uplo, double diag_add, void* ws, size_t ws_bytes) {
  if (m < 0 || n < 0 || k < 0) return QDWHP_ERR_ARG;
  if (m == 0 || n == 0) return QDWHP_OK;
  if (m > (1 << 24) || n > (1 << 24) || k > (1 << 24)) return QDWHP_ERR_ARG;
  if (k == 0) return gemm(st, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, uplo, diag_add);
  if (ws == nullptr || ws_bytes < gemm_ozaki_ws_bytes(m, n, k)) return QDWHP_ERR_NOMEM;
  QDWHP_TRY(upload_pairs());
  const int mp = ceil_to(m, kOzBM), np = ceil_to(n, kOzBN), kp = ceil_to(k, kOzKPad);
  unsigned short* Asl = (unsigned short*)ws;
  unsigned short* Bsl = Asl + (size_t)kOzS * mp * kp;
  int* ea = (int*)(Bsl + (size_t)kOzS * np * kp);
  int* eb = ea + mp;
  int* err = eb + np;   // set by the tcgen05 kernel if a bounded wait gave up (its tile is then NaN)
  // exponents: op(A) rows (r contiguous iff A is not transposed), op(B) columns (j contiguous
  // iff B is transposed)
  oz_init_exp_kernel<<<ceil_div(mp + np, 256), 256, 0, st>>>(mp + np, ea);
  QDWHP_LAUNCH_CHECK();
  oz_exp_kernel<<<dim3(ceil_div(m, 32), ceil_div(k, 32)), 256, 0, st>>>((int)m, (int)k, A, lda, ta ? 0 : 1, ea);
  QDWHP_LAUNCH_CHECK();
  oz_exp_kernel<<<dim3(ceil_div(n, 32), ceil_div(k, 32)), 256, 0, st>>>((int)n, (int)k, B, ldb, tb ? 1 : 0, eb);
  QDWHP_LAUNCH_CHECK();
  oz_split_kernel<<<dim3(mp / 32, kp / 32), 256, 0, st>>>((int)m, (int)k, mp, kp, A, lda, ta ? 0 : 1, ea, Asl);
  QDWHP_LAUNCH_CHECK();
  oz_split_kernel<<<dim3(np / 32, kp / 32), 256, 0, st>>>((int)n, (int)k, np, kp, B, ldb, tb ? 1 : 0, eb, Bsl);
  QDWHP_LAUNCH_CHECK();
  const double flops = (uplo == LOWER) ? (double)n * (n + 1) * k : 2.0 * m * n * k;
  int prof_slot = -1;
  if (gemm_prof_enabled()) {
    const double shape[5] = {(double)m, (double)n, (double)k, (double)(uplo == LOWER), -1.0};
    prof_slot = gemm_prof_start(st, flops, shape);
  }
  QDWHP_TRY(launch_umma_ws(st, m, n, kp, mp, np, Asl, Bsl, ea, eb, alpha, beta, C, ldc, uplo, diag_add, err));
  if (prof_slot >= 0) gemm_prof_stop(st, prof_slot);
  return QDWHP_OK;
}

}  // namespace qdwhp
