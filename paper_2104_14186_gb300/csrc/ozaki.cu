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
// FP32 accumulators of mma.sync m16n8k16 (bf16 x bf16 -> f32).  Each such product is scaled
// by its power of two and added into FP64 accumulators.  The pairs with s + t <= 12 are
// kept (60 of the 81).  The dropped pairs are a bias, not noise, where the digit products
// share a sign (a sum of squares): at most 6 K 63^2 2^-78 2^(e_i + f_j), below FP64 rounding
// for the K of this library (at s + t <= 11 it reached 1e-13 relative at K = 16384).  Pairs
// of one level s + t share the scale 2^(-6 (s + t)), so they share an FP32 accumulator as
// long as it holds at most 4224 digit products (exact); it is flushed into FP64 when the
// level changes or the budget would be exceeded.
//
// Layout: digit slices are stored as [slice][row][k_pad] bfloat16 with K contiguous (op(A)
// rows, op(B) columns), zero-padded to the CTA tile; the GEMM streams a (slice pair, K block)
// sequence through a 3-stage cp.async pipeline and ldmatrix.
#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>

#include "internal.h"

namespace qdwhp {

namespace {

constexpr int kOzS = 9;          // digits per entry
constexpr int kOzBeta = 6;       // bits per digit
constexpr int kOzT = 12;         // keep digit pairs with s + t <= kOzT (1-based)
constexpr int kOzBudget = 4224;  // FP32 exactness: at most this many digit products (each
                                 // < 2^12 in magnitude) in one accumulator: 4224 * 63^2 < 2^24
constexpr int kOzBM = 128, kOzBN = 128, kOzBK = 32;   // kOzBN: padding of op(B) (either tile divides it)
constexpr int kOzLd = kOzBK + 8; // smem row stride (bf16): 80 bytes, conflict-free ldmatrix
constexpr int kOzThreads = 256;
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

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One CTA: a 128 x BN tile of C, 8 warps of (16 MT) x 32 (MT x 4 mma tiles of 16 x 8):
//   MT = 4: 2 x 4 warps, BN = 128 (16 mma per 6 ldmatrix.x4 per 16-deep step), 3 stages;
//   MT = 2: 4 x 2 warps, BN = 64 (more CTAs for narrow products; two CTAs fit an SM), 3 stages.
// The exact FP32 digit products live in registers; their FP64 sums live in shared memory,
// 16 MT doubles per thread at index f * 256 + thread, touched only by that thread.
template <int MT>
struct OzCfg {
  static constexpr int kWarpsM = kOzBM / (16 * MT);
  static constexpr int kWarpsN = 8 / kWarpsM;
  static constexpr int kBN = kWarpsN * 32;
  static constexpr int kStages = 3;
  static constexpr size_t kSmemStages = (size_t)kStages * (kOzBM + kBN) * kOzLd * sizeof(unsigned short);
  static constexpr size_t kSmemBytes = kSmemStages + (size_t)16 * MT * kOzThreads * sizeof(double);
};

template <int MT>
__global__ void __launch_bounds__(kOzThreads, 1) oz_gemm_kernel(int M, int N, int k_pad, int rows_a_pad,
                                                                int rows_b_pad, const unsigned short* __restrict__ Asl,
                                                                const unsigned short* __restrict__ Bsl,
                                                                const int* __restrict__ ea,
                                                                const int* __restrict__ eb, double alpha, double beta,
                                                                double* C, int64_t ldc, int uplo, double diag_add) {
  using Cfg = OzCfg<MT>;
  constexpr int BN = Cfg::kBN, STAGES = Cfg::kStages;
  extern __shared__ __align__(128) unsigned char oz_smem[];
  unsigned short* sA = reinterpret_cast<unsigned short*>(oz_smem);
  unsigned short* sB = sA + (size_t)STAGES * kOzBM * kOzLd;
  double* acc64 = reinterpret_cast<double*>(oz_smem + Cfg::kSmemStages);
  const int bm = blockIdx.y, bn = blockIdx.x;
  const int m0 = bm * kOzBM, n0 = bn * BN;
  if (uplo == LOWER && m0 + kOzBM <= n0) return;   // tile strictly above the diagonal
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp % Cfg::kWarpsM, wn = warp / Cfg::kWarpsM;
  const int nkb = k_pad / kOzBK;
  const int npairs = c_pairs.npairs;
  const int total = npairs * nkb;
  const size_t slice_a = (size_t)rows_a_pad * k_pad, slice_b = (size_t)rows_b_pad * k_pad;

  // the (pair, K block) of the next stage to load, advanced incrementally
  int lp = 0, lkb = 0;
  auto load_next = [&](int buf) {
    const unsigned short* As = Asl + (size_t)c_pairs.s[lp] * slice_a + (size_t)m0 * k_pad + lkb * kOzBK;
    const unsigned short* Bs = Bsl + (size_t)c_pairs.t[lp] * slice_b + (size_t)n0 * k_pad + lkb * kOzBK;
    unsigned short* da = sA + (size_t)buf * kOzBM * kOzLd;
    unsigned short* db = sB + (size_t)buf * BN * kOzLd;
#pragma unroll
    for (int q = 0; q < 2; ++q) {   // A: 128 rows x 4 chunks of 16 bytes
      const int c = tid + kOzThreads * q;
      const int row = c >> 2, ch = c & 3;
      cp_async16(da + row * kOzLd + ch * 8, As + (size_t)row * k_pad + ch * 8);
    }
#pragma unroll
    for (int q = 0; q < BN / 64; ++q) {   // B: BN rows x 4 chunks
      const int c = tid + kOzThreads * q;
      const int row = c >> 2, ch = c & 3;
      cp_async16(db + row * kOzLd + ch * 8, Bs + (size_t)row * k_pad + ch * 8);
    }
    if (++lkb == nkb) {
      lkb = 0;
      ++lp;
    }
  };

  float acc[MT][4][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
#pragma unroll 8
  for (int f = 0; f < 16 * MT; ++f) acc64[f * kOzThreads + tid] = 0.0;

#pragma unroll
  for (int st = 0; st < STAGES - 1; ++st) {
    if (st < total) load_next(st);
    cp_async_commit();
  }
  int cp = 0, ckb = 0;   // (pair, K block) being computed
  int terms = 0;         // digit products in the FP32 accumulators since the last flush
  for (int step = 0; step < total; ++step) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    if (step + STAGES - 1 < total) load_next((step + STAGES - 1) % STAGES);
    cp_async_commit();
    const int buf = step % STAGES;
    const unsigned short* a_s = sA + (size_t)buf * kOzBM * kOzLd;
    const unsigned short* b_s = sB + (size_t)buf * BN * kOzLd;
#pragma unroll
    for (int kk = 0; kk < kOzBK; kk += 16) {
      unsigned af[MT][4];
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int row = wm * 16 * MT + mt * 16 + (lane & 15);
        const int col = kk + ((lane >> 4) << 3);
        ldmatrix_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3], a_s + row * kOzLd + col);
      }
      unsigned bfr[4][2];
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        const int nrow = wn * 32 + np * 16 + (lane & 7) + ((lane >> 4) << 3);
        const int col = kk + (((lane >> 3) & 1) << 3);
        unsigned r0, r1, r2, r3;
        ldmatrix_x4(r0, r1, r2, r3, b_s + nrow * kOzLd + col);
        bfr[2 * np][0] = r0;
        bfr[2 * np][1] = r1;
        bfr[2 * np + 1][0] = r2;
        bfr[2 * np + 1][1] = r3;
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bfr[nt][0], bfr[nt][1]);
    }
    // flush the exact FP32 sums into FP64 when the next step changes level or would exceed
    // the exactness budget (the same decision in every thread)
    terms += kOzBK;
    int np_ = cp, nkb_ = ckb + 1;
    if (nkb_ == nkb) {
      nkb_ = 0;
      ++np_;
    }
    if (np_ >= npairs || c_pairs.lev[np_] != c_pairs.lev[cp] || terms + kOzBK > kOzBudget) {
      terms = 0;
      const double sc = c_pairs.scale[cp];
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            double* slot = acc64 + ((i * 4 + j) * 4 + q) * kOzThreads + tid;
            *slot = fma((double)acc[i][j][q], sc, *slot);
            acc[i][j][q] = 0.f;
          }
    }
    if (++ckb == nkb) {
      ckb = 0;
      ++cp;
    }
  }
  cp_async_wait<0>();

  // epilogue: C = alpha 2^(e_i + f_j) acc + beta C (+ diag_add on the diagonal)
  const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int i = m0 + wm * 16 * MT + mt * 16 + g + 8 * half;
      if (i >= M) continue;
      const int e_i = ea[i];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int j = n0 + wn * 32 + nt * 8 + 2 * t4 + cc;
          if (j >= N) continue;
          if (uplo == LOWER && i < j) continue;
          const int f_j = eb[j];
          double v;
          if (e_i == kExpNonfinite || f_j == kExpNonfinite) {
            v = __longlong_as_double(0x7ff8000000000000ll);
          } else if (e_i == kExpEmpty || f_j == kExpEmpty) {
            v = 0.0;
          } else {
            v = alpha * ldexp(acc64[((mt * 4 + nt) * 4 + 2 * half + cc) * kOzThreads + tid], e_i + f_j);
          }
          double* cptr = C + i + (int64_t)j * ldc;
          if (beta != 0.0) v = fma(beta, *cptr, v);
          if (i == j) v += diag_add;
          *cptr = v;
        }
      }
    }
  }
}

template <int MT>
qdwhp_status launch_oz(cudaStream_t st, int64_t m, int64_t n, int kp, int mp, int np, const unsigned short* Asl,
                       const unsigned short* Bsl, const int* ea, const int* eb, double alpha, double beta, double* C,
                       int64_t ldc, Uplo uplo, double diag_add) {
  using Cfg = OzCfg<MT>;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(oz_gemm_kernel<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Cfg::kSmemBytes);
  });
  QDWHP_CUDA_TRY(attr_err);
  dim3 grid(np / Cfg::kBN, mp / kOzBM);
  oz_gemm_kernel<MT><<<grid, kOzThreads, Cfg::kSmemBytes, st>>>((int)m, (int)n, kp, mp, np, Asl, Bsl, ea, eb, alpha,
                                                                beta, C, ldc, (int)uplo, diag_add);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

int ceil_to(int64_t a, int b) { return (int)(((a + b - 1) / b) * b); }

std::once_flag g_pairs_once;
qdwhp_status g_pairs_status = QDWHP_OK;

qdwhp_status upload_pairs() {
  std::call_once(g_pairs_once, [] {
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
    if (cudaMemcpyToSymbol(c_pairs, &t, sizeof(t)) != cudaSuccess) g_pairs_status = QDWHP_ERR_CUDA;
  });
  return g_pairs_status;
}

}  // namespace

size_t gemm_ozaki_ws_bytes(int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  const size_t mp = ceil_to(m, kOzBM), np = ceil_to(n, kOzBN), kp = ceil_to(k, kOzBK);
  return (size_t)kOzS * (mp + np) * kp * 2 + (mp + np) * sizeof(int) + 1024;
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
  const int mp = ceil_to(m, kOzBM), np = ceil_to(n, kOzBN), kp = ceil_to(k, kOzBK);
  unsigned short* Asl = (unsigned short*)ws;
  unsigned short* Bsl = Asl + (size_t)kOzS * mp * kp;
  int* ea = (int*)(Bsl + (size_t)kOzS * np * kp);
  int* eb = ea + mp;
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
  // 128 x 128 tiles when they fill the GPU twice over, else 128 x 64 (twice the CTAs)
  int dev = 0, sms = kNumSMs;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t big_tiles = (int64_t)(mp / kOzBM) * (np / 128) / (uplo == LOWER ? 2 : 1);
  if (big_tiles >= 2 * sms) {
    QDWHP_TRY(launch_oz<4>(st, m, n, kp, mp, np, Asl, Bsl, ea, eb, alpha, beta, C, ldc, uplo, diag_add));
  } else {
    QDWHP_TRY(launch_oz<2>(st, m, n, kp, mp, np, Asl, Bsl, ea, eb, alpha, beta, C, ldc, uplo, diag_add));
  }
  if (prof_slot >= 0) gemm_prof_stop(st, prof_slot);
  return QDWHP_OK;
}

}  // namespace qdwhp
