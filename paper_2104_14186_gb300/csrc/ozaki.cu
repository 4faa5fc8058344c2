// FP64 GEMM emulated on the BF16 tensor cores by the Ozaki splitting scheme
// (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication and its applications", Numer. Algorithms
// 59 (2012); as run on low-precision tensor cores by Mukunoki, Ozaki, Ogita, Imamura, 2020).
// Not part of the paper's method: a faster route to FP64-accurate products on a part whose
// FP64 pipe is ~1/600 of its BF16 tensor rate.
//
// Each row i of op(A) is scaled by 2^-e_i (e_i: binary exponent of the row's largest
// magnitude, so every entry lies in (-1, 1)) and rounded to a 53-bit fixed-point integer X,
// written in base 2^6 as 9 balanced signed digits D_1..D_9 (|D| <= 32: exact in bfloat16):
// X = sum_s D_s 2^(6 (9 - s)), so the entry is 2^(e_i + 1) sum_s D_s 2^(-6 s).  Columns of op(B)
// are split the same way with exponents f_j.  Then
//     C_ij = 2^(e_i + f_j + 2) sum_{s,t} 2^(-6 (s + t)) (D^A_s D^B_t)_ij ,
// where every digit product D^A_s D^B_t is an exact integer matrix product: each term is at
// most 2^10 in magnitude, so a sum of up to 2^14 terms stays within 2^24 and is exact in the
// FP32 accumulators of the tensor cores (bf16 x bf16 -> f32).  Each such sum is scaled by its
// power of two and added into FP64 accumulators.  The pairs with s + t <= 12 are kept (60 of
// the 81).  The dropped pairs are a bias, not noise, where the digit products share a sign (a
// sum of squares): at most 6 K 2^10 2^-78 2^(e_i + f_j + 2), far below the K u 2^(e_i + f_j)
// rounding bound of an FP64 dot product of length K.  The 53-bit rounding of an entry is at
// most 2^-54 2^(e_i + 1) <= 2^-53 times its row's largest magnitude.  Pairs of one level s + t
// share the scale 2^(-6 (s + t)), so they share an FP32 accumulator while it holds at most 2^14
// digit products per entry; the schedule (oz_schedule.h) flushes it into FP64 before that.
//
// Layout: digit slices are stored as [slice][row][k_pad] bfloat16 with K contiguous (op(A)
// rows, op(B) columns), zero-padded to 128-row blocks and 64-deep K steps; the product kernel
// (TMA + tcgen05, below) runs the schedule's 2 x 2 digit blocks, each K step loading up to two
// op(A) and two op(B) digit tiles into one stage of a 3-stage ring in shared memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>

#include "internal.h"
#include "oz_schedule.h"
#include "umma.cuh"

namespace qdwhp {

namespace {

constexpr int kOzBeta = 6;       // bits per digit
constexpr int kOzBM = 128, kOzBN = 128;   // row padding of the op(A) and op(B) digit slices
constexpr int kOzKPad = kOzStepK;         // K padding of the digit slices (one K step)
constexpr int kExpEmpty = -2000000000;   // no entry seen yet (row of zeros)
constexpr int kExpNonfinite = 1 << 20;   // a NaN or Inf in the row

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
  // |d| <= 32: exactly representable; round-to-nearest conversion is exact
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
    long long X53 = 0;
    if (e != kExpEmpty && e != kExpNonfinite && v != 0.0) {
      // |v| 2^-e < 1; scaled by 2^53 it is below 2^53; rounding to an integer moves it by <= 1/2
      X53 = llrint(ldexp(v, 53 - e));
    }
    const unsigned long long U = (unsigned long long)(X53 < 0 ? -X53 : X53);
    const int sgn = X53 < 0 ? -1 : 1;
    unsigned short* o = out + (size_t)r * k_pad + l;
    // balanced digits, least significant first: a 6-bit group of 32 or more becomes group - 64
    // with a carry into the next group; the top group (bits 48..52, < 32) takes the last carry
    int carry = 0;
#pragma unroll
    for (int s = kOzS - 1; s >= 1; --s) {
      int d = (int)((U >> (kOzBeta * (kOzS - 1 - s))) & ((1u << kOzBeta) - 1)) + carry;
      carry = d >= 32 ? 1 : 0;
      d -= 64 * carry;
      o[(size_t)s * slice] = bf16_bits_of_small_int(sgn * d);
    }
    o[0] = bf16_bits_of_small_int(sgn * ((int)(U >> (kOzBeta * (kOzS - 1))) + carry));
  }
}

// ---- the digit-product kernel (TMA + tcgen05, warp-specialised, schedule-driven) ----
//
// One CTA computes a 128 x 128 tile of C.  The digit products run on the 5th-generation tensor
// cores as tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = N = 128, K = 16), both operands read
// from shared memory through matrix descriptors: K-major, 128-byte swizzle, i.e. 8-row atoms of
// 1024 bytes with 16-byte chunk c of row r stored at chunk c ^ (r % 8), which is the layout the
// TMA engine writes for a 64 x 128 box with the 128-byte swizzle.  (32-deep steps with the
// 64-byte swizzle fit seven 32 KB stages, but ran the 4096^3 product a third slower.)
//
// Two threads walk the schedule (oz_schedule.h).
// * Warp 9 (one thread) copies, for every K step of an item, the item's digit tiles into a
//   64 KB stage (op(A) digits into tile slots 0-1, op(B) digits into 2-3; the stage's "full"
//   mbarrier counts the bytes) as soon as the stage's "empty" mbarrier says the MMAs of its
//   previous step are done.
// * Warp 8 (one thread), once a stage is full, issues the item's pair products into their
//   tensor-memory slots (four 128-column FP32 accumulators) and commits them to the stage's
//   "empty" mbarrier.  It never waits on its own MMAs: a single thread that also refilled the
//   ring had to, so copy latency and MMA time added up (9.6 against 7.5 ms for the 4096^3
//   product).  After an item it commits the "ready" mbarrier of every slot the schedule
//   flushes there; before writing a reused slot it waits on that slot's "free" mbarrier.
// * Warps 0-7 only flush: for each flush of the schedule they wait (sleeping between polls)
//   on the slot's "ready", read its FP32 sums (tcgen05.ld), add them times 2^(-6 level) into
//   their FP64 registers and arrive on "free".
// Every wait is bounded: on a timeout the tile is written as NaN and err is set.
constexpr int kOzThreads = 320;
constexpr int kOzStages = 3;
constexpr uint32_t kOzTileBytes = 128 * kOzStepK * 2;      // 16 KB: 128 rows x 64 K of one digit
constexpr uint32_t kOzStageBytes = 4 * kOzTileBytes;       // op(A) tiles 0-1, op(B) tiles 2-3
constexpr size_t kOzSmemBytes = (size_t)kOzStages * kOzStageBytes + 1024;
constexpr int kOzTmemCols = kOzSlots * 128;
constexpr int kOzGroupM = 8;   // tile rows per band of the tile order (152 resident CTAs: 8 x 19 tiles)

__global__ void __launch_bounds__(kOzThreads, 1)
    oz_umma_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ OzSchedule sch, int M, int N, int ntm, int ntn, int kb0,
                   const int* __restrict__ ea, const int* __restrict__ eb, double alpha, double beta, double* C,
                   int64_t ldc, int uplo, double diag_add, int* err) {
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t bar_full[kOzStages], bar_empty[kOzStages];
  __shared__ __align__(8) uint64_t bar_ready[kOzSlots], bar_free[kOzSlots], bar_done;
  __shared__ int s_abort, s_zero;
  // tile order: bands of kOzGroupM tile rows, column by column inside a band, so that the CTAs
  // resident at one time share their op(A) and op(B) digit tiles in L2
  const int band = (int)blockIdx.x / (kOzGroupM * ntn), local = (int)blockIdx.x - band * kOzGroupM * ntn;
  const int gm = min(kOzGroupM, ntm - band * kOzGroupM);
  const int m0 = (band * kOzGroupM + local % gm) * 128, n0 = (local / gm) * 128;
  if (uplo == LOWER && m0 + 128 <= n0) return;   // tile strictly above the diagonal
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(umma::smem_addr(&tmem_base)),
                 "r"(kOzTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 256) {
    for (int s = 0; s < kOzStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_addr(&bar_full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_addr(&bar_empty[s])));
    }
    for (int x = 0; x < kOzSlots; ++x) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma::smem_addr(&bar_ready[x])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(umma::smem_addr(&bar_free[x])));
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
  int issued = 0;   // steps whose copy the producer issued

  if (warp >= 8) {
    if (lane == 0) {
      const uint32_t sbase = umma::smem_addr(smem);
      int total = 0;
      for (int it = 0; it < sch.nitems; ++it) total += oz_item_steps(sch, it);
      if (warp == 9) {
        // producer: step j goes to stage j % kOzStages once the MMAs of step j - kOzStages are done
        int li = 0, lks = 0;   // the next step to load: item li, its step lks
        for (int j = 0; j < total; ++j) {
          const int stage = j % kOzStages;
          if (j >= kOzStages && !umma::mbar_wait_or_abort(umma::smem_addr(&bar_empty[stage]),
                                                          (uint32_t)((j / kOzStages - 1) & 1), abort_flag)) {
            ok = false;
            break;
          }
          const int at = sch.atile[li], bt = sch.btile[li];
          const bool a2 = (at >> 4) != 0xF, b2 = (bt >> 4) != 0xF;
          const uint32_t bar = umma::smem_addr(&bar_full[stage]);
          const uint32_t bytes = (uint32_t)(2 + (a2 ? 1 : 0) + (b2 ? 1 : 0)) * kOzTileBytes;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
          const int kc = (kb0 + sch.chunk[li] * sch.clen + lks) * kOzStepK;
          const uint32_t d = sbase + (uint32_t)stage * kOzStageBytes;
          umma::tma_load_3d(d, &mapA, kc, m0, at & 15, bar);
          if (a2) umma::tma_load_3d(d + kOzTileBytes, &mapA, kc, m0, at >> 4, bar);
          umma::tma_load_3d(d + 2 * kOzTileBytes, &mapB, kc, n0, bt & 15, bar);
          if (b2) umma::tma_load_3d(d + 3 * kOzTileBytes, &mapB, kc, n0, bt >> 4, bar);
          issued = j + 1;
          if (++lks == oz_item_steps(sch, li)) {
            lks = 0;
            ++li;
          }
        }
        if (!ok) *abort_flag = 1;
      } else {
        // MMA issuer: never waits on its own MMAs, so the tensor pipe is fed as far ahead as the
        // copies allow
        const uint32_t idesc = umma::idesc_bf16_f32(128, 128);
        int ci = 0, cks = 0, fp = 0;
        uint32_t nf = 0;   // flushes committed per slot, 8 bits each
        for (int step = 0; step < total && ok; ++step) {
          const int stage = step % kOzStages;
          if (!umma::mbar_wait_or_abort(umma::smem_addr(&bar_full[stage]), (uint32_t)((step / kOzStages) & 1),
                                        abort_flag)) {
            ok = false;
            break;
          }
          if (cks == 0) {
            // reused slots: their last flush has read them out
            const int wm = sch.ctl[ci] & 15;
            for (int x = 0; x < kOzSlots && ok; ++x)
              if ((wm >> x) & 1) {
                const uint32_t cnt = (nf >> (8 * x)) & 255u;
                if (!umma::mbar_wait_or_abort(umma::smem_addr(&bar_free[x]), (cnt - 1u) & 1u, abort_flag)) ok = false;
              }
            if (!ok) break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t st_base = sbase + (uint32_t)stage * kOzStageBytes;
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int pc = sch.pair[ci][p];
            if (!(pc & 0x80)) continue;
            const uint32_t a0 = st_base + (uint32_t)(pc & 1) * kOzTileBytes;
            const uint32_t b0 = st_base + (uint32_t)(2 + ((pc >> 1) & 1)) * kOzTileBytes;
            const uint32_t dcol = tmem + (uint32_t)(((pc >> 2) & 3) * 128);
            const bool fresh = (pc & 0x10) && cks == 0;
#pragma unroll
            for (int kk = 0; kk < kOzStepK / 16; ++kk)   // 32-byte K steps inside the 128-byte rows
              umma::mma_bf16(dcol, umma::desc_sw128(a0 + kk * 32), umma::desc_sw128(b0 + kk * 32), idesc,
                             (fresh && kk == 0) ? 0u : 1u);
          }
          umma::commit(umma::smem_addr(&bar_empty[stage]));
          if (++cks == oz_item_steps(sch, ci)) {
            const int nfl = (sch.ctl[ci] >> 4) & 7;
            for (int f = 0; f < nfl; ++f) {
              const int x = sch.flush[fp++] & 3;
              umma::commit(umma::smem_addr(&bar_ready[x]));
              nf += 1u << (8 * x);
            }
            cks = 0;
            ++ci;
          }
        }
        if (!ok) *abort_flag = 1;
        umma::commit(umma::smem_addr(&bar_done));   // every MMA issued so far
        // the tensor memory is freed below only after those MMAs are done (bounded)
        umma::mbar_wait_or_abort(umma::smem_addr(&bar_done), 0, &s_zero);
      }
    }
    __syncwarp();
  } else {
    // flush warps: row (warp % 4) * 32 + lane, columns (warp / 4) * 64 + [0, 64) of every slot
    double acc64[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) acc64[j] = 0.0;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t col_base = (uint32_t)((warp >> 2) * 64);
    uint32_t nfw = 0;   // flushes done per slot, 8 bits each
    for (int j = 0; j < sch.nflush && ok; ++j) {
      const int fl = sch.flush[j], x = fl & 3, lev = fl >> 2;
      const uint32_t cnt = (nfw >> (8 * x)) & 255u;
      if (!umma::mbar_wait_sleep_or_abort(umma::smem_addr(&bar_ready[x]), cnt & 1u, abort_flag)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const double sc = __longlong_as_double((long long)(1023 - kOzBeta * lev) << 52);   // 2^(-6 lev), exact
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t v[32];
        umma::tmem_ld32(tmem + lane_base + (uint32_t)(x * 128) + col_base + (uint32_t)(32 * h), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int c = 0; c < 32; ++c) acc64[32 * h + c] = fma((double)__uint_as_float(v[c]), sc, acc64[32 * h + c]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_addr(&bar_free[x])) : "memory");
      nfw += 1u << (8 * x);
    }
    if (!ok) *abort_flag = 1;
    if (!umma::mbar_wait_sleep_or_abort(umma::smem_addr(&bar_done), 0, abort_flag)) ok = false;
    // epilogue: C = alpha 2^(e_i + f_j + 2) acc + beta C (+ diag_add on the diagonal)
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
          v = alpha * ldexp(acc64[c], e_i + f_j + 2);
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
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzTmemCols));
  if (warp == 9 && lane == 0 && *abort_flag) {
    // after a give-up anywhere in the CTA: the last copy into each stage lands before the CTA's
    // shared memory is released (bounded)
    for (int j = issued > kOzStages ? issued - kOzStages : 0; j < issued; ++j)
      umma::mbar_wait_or_abort(umma::smem_addr(&bar_full[j % kOzStages]), (uint32_t)((j / kOzStages) & 1), &s_zero);
  }
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

// Schedules by number of K steps, built once per size and kept for the process.
const OzSchedule* schedule_for(int nsteps) {
  static std::mutex mu;
  static std::map<int, std::unique_ptr<OzSchedule>> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(nsteps);
  if (it != cache.end()) return it->second.get();
  std::unique_ptr<OzSchedule> s(new OzSchedule);
  if (!oz_build_schedule(nsteps, s.get())) return nullptr;
  return (cache[nsteps] = std::move(s)).get();
}

qdwhp_status launch_oz(cudaStream_t st, int64_t m, int64_t n, int kp, int mp, int np, const unsigned short* Asl,
                       const unsigned short* Bsl, const int* ea, const int* eb, double alpha, double beta, double* C,
                       int64_t ldc, Uplo uplo, double diag_add, int* err) {
  static PerDeviceOnce attr;
  QDWHP_CUDA_TRY(attr.run([] {
    return cudaFuncSetAttribute(oz_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmemBytes);
  }));
  CUtensorMap mapA, mapB;
  QDWHP_TRY(umma::slice_map(&mapA, Asl, kOzS, mp, kp));
  QDWHP_TRY(umma::slice_map(&mapB, Bsl, kOzS, np, kp));
  const int ntm = mp / 128, ntn = np / 128;
  const dim3 grid((unsigned)(ntm * ntn));
  const int nsteps = kp / kOzStepK;
  // K beyond one schedule's reach: later launches add onto C
  for (int kb0 = 0; kb0 < nsteps; kb0 += kOzMaxSteps) {
    const int ns = nsteps - kb0 < kOzMaxSteps ? nsteps - kb0 : kOzMaxSteps;
    const OzSchedule* sch = schedule_for(ns);
    if (sch == nullptr) {
      set_error_message("no digit-product schedule for this K");
      return QDWHP_ERR_ARG;
    }
    const bool first = kb0 == 0;
    oz_umma_kernel<<<grid, kOzThreads, kOzSmemBytes, st>>>(mapA, mapB, *sch, (int)m, (int)n, ntm, ntn, kb0, ea, eb, alpha,
                                                           first ? beta : 1.0, C, ldc, (int)uplo,
                                                           first ? diag_add : 0.0, err);
    QDWHP_LAUNCH_CHECK();
  }
  return QDWHP_OK;
}

int ceil_to(int64_t a, int b) { return (int)(((a + b - 1) / b) * b); }

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
  QDWHP_TRY(launch_oz(st, m, n, kp, mp, np, Asl, Bsl, ea, eb, alpha, beta, C, ldc, uplo, diag_add, err));
  if (prof_slot >= 0) gemm_prof_stop(st, prof_slot);
  return QDWHP_OK;
}

}  // namespace qdwhp
