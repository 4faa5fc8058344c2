// Blocked Householder QR (unpivoted) and explicit columns of Q.
//
// Used for the extraction step (Algorithm 1 step 3, Algorithm 2 step 3), the
// QR-based QDWH step (eq. practical-polar-qr) and the orthonormalisation of the
// count-to-threshold subspace.  Reflectors follow the LAPACK convention
// H = I - tau v v^T with v_1 = 1, and each kQRNB-wide panel is
// accumulated into the compact WY form Q_p = I - V T V^T (T upper triangular).
// Two levels: a panel updates only the rest of its 256-column outer block; the outer
// block's T (merged from its eight panel T's through the Gram matrix G = V^T V:
// T_{1:q+1} = [T_{1:q}, -T_{1:q} G(1:q, q+1) T_{q+1}; 0, T_{q+1}]) then updates the
// trailing matrix and forms Q with products of inner dimension 256.
//
// One SM does only a few FP64 flops per clock on this part, so a panel factored by
// a single CTA would be ~100x slower than the chip.  The panel kernel is therefore
// a cooperative launch over up to kPanelCTAs CTAs: each CTA keeps its slice of
// rows in shared memory, and the column norms and the reflector-application dot
// products are reduced across CTAs through global partials with one grid-wide
// barrier per column (the squared norm and the dot products with the later columns
// are summed together; the reflector's w_c = v^T x_c follows from them locally).  Partials are summed in CTA order, so the factorisation is
// reproducible run to run.  The trailing update and the formation of Q are GEMMs.
#include <cooperative_groups.h>

#include <mutex>

#include "internal.h"

namespace cg = cooperative_groups;

namespace qdwhp {

namespace {

constexpr int NB = kQRNB;          // panel width (32)
constexpr int NBO = kQROuter;      // outer block width (256 = 8 panels)
constexpr size_t kQRSplitCap = size_t(4) << 20;   // split-K scratch of the trailing products (doubles)
constexpr int kPanelThreads = 256;
constexpr int kPanelCTAs = 96;
constexpr int kPartStride = NB + 1;

struct PanelArgs {
  int R;            // rows of the panel (from its diagonal down)
  int jb;           // width
  double* P;        // A(j, j)
  int64_t lda;
  double* V;        // explicit reflectors, R x jb, ld ldv
  int64_t ldv;
  double* T;        // jb x jb (ld NB)
  double* tau;      // jb
  double* diagR;    // jb
  double* part;     // 2 x kPanelCTAs x kPartStride (double-buffered by column parity)
  double* gram;     // (gridDim.x + 1) * NB * NB: per-CTA partials, then the totals
  double* row_slot;   // 2 x NB doubles: row i of the panel, published by its owner
};

__global__ void __launch_bounds__(kPanelThreads) panel_qr_kernel(PanelArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double s[];          // local rows: s[r + c * rpc]
  __shared__ double red8[8][NB];
  __shared__ double wsh[NB];
  __shared__ double rowv[NB];
  __shared__ double taus[NB], betas[NB];

  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int R = a.R, jb = a.jb;
  const int rpc = (R + G - 1) / G;
  const int r0 = b * rpc;
  const int nr = max(0, min(R, r0 + rpc) - r0);

  for (int e = tid; e < rpc * NB; e += blockDim.x) {
    const int r = e % rpc, c = e / rpc;
    s[e] = (r < nr && c < jb) ? a.P[(r0 + r) + (int64_t)c * a.lda] : 0.0;
  }
  __syncthreads();

  for (int i = 0; i < jb; ++i) {
    // Partials and the published row are double-buffered by column parity: with one
    // barrier per column, a CTA may already write column i+1's partials while another
    // still reads column i's.
    double* part = a.part + (i & 1) * (kPanelCTAs * kPartStride);
    double* row_slot = a.row_slot + (i & 1) * NB;
    // Phase A (one grid barrier per column): each CTA sums, over its rows below row i,
    // x_r,i^2 and x_r,i x_r,c for the columns c > i; the owner of row i publishes the
    // row-i entries (alpha = x_i,i and x_i,c).
    {
      const int c = tid % NB, grp = tid / NB;   // 8 row groups x 32 columns
      double p = 0.0;
      if (c >= i && c < jb) {
        for (int r = grp; r < nr; r += 8) {
          if (r0 + r > i) p += s[r + i * rpc] * s[r + c * rpc];
        }
      }
      red8[grp][c] = p;
    }
    __syncthreads();
    if (tid < NB) {
      double p = 0.0;
#pragma unroll
      for (int g8 = 0; g8 < 8; ++g8) p += red8[g8][tid];
      // slot i holds the squared norm, slots c > i the dot products
      if (tid >= i && tid < jb) part[b * kPartStride + tid] = p;
      if (i >= r0 && i < r0 + nr && tid >= i && tid < jb) row_slot[tid] = s[(i - r0) + tid * rpc];
    }
    grid.sync();

    // Phase B: every CTA sums the partials in the same fixed order (8 groups of CTAs per
    // slot) and forms the reflector: beta = -sign(alpha) sqrt(alpha^2 + ss), tau = (beta -
    // alpha) / beta, v = [1; x(i+1:) / (alpha - beta)], and w_c = v^T x_c = x_i,c + e_c / (alpha - beta).
    {
      const int c = tid % NB, grp = tid / NB;
      double w = 0.0;
      if (c >= i && c < jb) {
#pragma unroll 4
        for (int g = grp; g < G; g += 8) w += part[g * kPartStride + c];
      }
      red8[grp][c] = w;
    }
    __syncthreads();
    if (tid < NB) {
      double w = 0.0;
#pragma unroll
      for (int g8 = 0; g8 < 8; ++g8) w += red8[g8][tid];
      wsh[tid] = w;                              // wsh[i] = ss, wsh[c > i] = e_c
      rowv[tid] = (tid >= i && tid < jb) ? row_slot[tid] : 0.0;
    }
    __syncthreads();
    const double ss = wsh[i];
    const double alpha = rowv[i];
    double beta, tau_i, scale;
    if (ss == 0.0) {
      beta = alpha;
      tau_i = 0.0;
      scale = 0.0;
    } else {
      beta = -copysign(sqrt(alpha * alpha + ss), alpha);
      tau_i = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    __syncthreads();
    if (tid == 0) {
      taus[i] = tau_i;
      betas[i] = beta;
    }
    if (tid < NB && tid > i && tid < jb) wsh[tid] = rowv[tid] + scale * wsh[tid];
    for (int r = tid; r < nr; r += blockDim.x) {
      const int rg = r0 + r;
      if (rg > i) s[r + i * rpc] *= scale;
      else if (rg == i) s[r + i * rpc] = 1.0;
    }
    __syncthreads();
    // Phase C: x_c -= tau w_c v on rows >= i for c > i (local rows only).
    if (tau_i != 0.0) {
      for (int e = tid; e < nr * NB; e += blockDim.x) {
        const int r = e % nr, c = e / nr;
        if (c > i && c < jb && r0 + r >= i) s[r + c * rpc] -= tau_i * wsh[c] * s[r + i * rpc];
      }
    }
    __syncthreads();
  }

  // Gram matrix V^T V of the explicit reflectors (for T), partial per CTA.
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int p = e % NB, q = e / NB;
    double acc = 0.0;
    if (p < jb && q < jb) {
      for (int r = 0; r < nr; ++r) {
        const int rg = r0 + r;
        const double vp = (rg > p) ? s[r + p * rpc] : (rg == p ? 1.0 : 0.0);
        const double vq = (rg > q) ? s[r + q * rpc] : (rg == q ? 1.0 : 0.0);
        acc += vp * vq;
      }
    }
    a.gram[(size_t)b * NB * NB + e] = acc;
  }
  // Write back: R above the diagonal and beta on it, compact v below; explicit V.
  for (int e = tid; e < nr * jb; e += blockDim.x) {
    const int r = e % nr, c = e / nr;
    const int rg = r0 + r;
    const double v = s[r + c * rpc];
    double* ap = a.P + rg + (int64_t)c * a.lda;
    double* vp = a.V + rg + (int64_t)c * a.ldv;
    if (rg < c) {
      *ap = v;
      *vp = 0.0;
    } else if (rg == c) {
      *ap = betas[c];
      *vp = 1.0;
    } else {
      *ap = v;
      *vp = v;
    }
  }
  grid.sync();

  // Sum the per-CTA Gram partials: CTA b owns entries [b*chunk, (b+1)*chunk).
  {
    const int chunk = (NB * NB + G - 1) / G;
    const int e0 = b * chunk, e1 = min(NB * NB, e0 + chunk);
    for (int e = e0 + tid; e < e1; e += blockDim.x) {
      double acc = 0.0;
#pragma unroll 4
      for (int g = 0; g < G; ++g) acc += a.gram[(size_t)g * NB * NB + e];
      a.gram[(size_t)G * NB * NB + e] = acc;
    }
  }
  grid.sync();

  if (b == 0) {
    // T (forward, columnwise): T_ii = tau_i, T(0:i, i) = -tau_i T(0:i, 0:i) (V^T v_i)(0:i).
    __shared__ double gsum[NB][NB + 1];
    __shared__ double Ts[NB][NB + 1];
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      gsum[e % NB][e / NB] = a.gram[(size_t)G * NB * NB + e];
      Ts[e % NB][e / NB] = 0.0;
    }
    __syncthreads();
    for (int i = 0; i < jb; ++i) {
      if (tid < i) {
        double acc = 0.0;
        for (int q = tid; q < i; ++q) acc += Ts[tid][q] * gsum[q][i];
        Ts[tid][i] = -taus[i] * acc;
      }
      if (tid == 0) Ts[i][i] = taus[i];
      __syncthreads();
    }
    for (int e = tid; e < NB * NB; e += blockDim.x) a.T[e] = Ts[e % NB][e / NB];
    if (tid < jb) {
      a.tau[tid] = taus[tid];
      a.diagR[tid] = betas[tid];
    }
  }
}

// CTAs of a panel of R rows: one per kTunePanelRows rows (64 unless tuned), at most kPanelCTAs.
int panel_ctas(int R) {
  const int rows = tune_value(kTunePanelRows, R);
  int g = (R + rows - 1) / rows;
  return std::max(1, std::min(g, kPanelCTAs));
}

size_t panel_smem_bytes(int R, int G) {
  const int rpc = (R + G - 1) / G;
  return (size_t)rpc * NB * sizeof(double);
}

qdwhp_status launch_panel(cudaStream_t st, PanelArgs& pa) {
  const int G = panel_ctas(pa.R);
  const size_t smem = panel_smem_bytes(pa.R, G);
  static PerDeviceOnce attr;
  QDWHP_CUDA_TRY(attr.run(
      [] { return cudaFuncSetAttribute(panel_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024); }));
  if (smem > 160 * 1024) return QDWHP_ERR_ARG;
  void* args[] = {&pa};
  return launch_cooperative((const void*)panel_qr_kernel, dim3(G), dim3(kPanelThreads), args, smem, st);
}

}  // namespace

// Split-K scratch of the trailing products: non-decreasing in n, so a scratch sized for n
// serves every narrower product.
size_t qr_splitk_elems(int64_t n) { return std::min((size_t)16 * NBO * std::max<int64_t>(n, 1), kQRSplitCap); }

size_t qr_to_elems(int64_t n) { return (size_t)ceil_div(std::max<int64_t>(n, 1), NBO) * NBO * NBO; }

size_t qr_scratch_elems(int64_t m, int64_t n) {
  const size_t wn = (size_t)NBO * std::max<int64_t>(n, 1);
  return 2 * wn + qr_splitk_elems(n) + 2 * (size_t)kPanelCTAs * kPartStride + (size_t)(kPanelCTAs + 1) * NB * NB +
         2 * NB + (size_t)NBO * NBO + (size_t)NBO * NB + 64;
  (void)m;
}

namespace {

// Rows of the reflectors of the columns [j, j + w): all of [j, m), or, for a factorisation with a
// band (the stacked [X; D] of a QR-based QDWH step, D diagonal, band = rows of X), only
// [j, band + j + w): the rows of D below are still zero in those columns.
int64_t active_rows(const QRFactors& f, int64_t j, int64_t w) {
  const int64_t end = f.band > 0 ? std::min<int64_t>(f.m, f.band + j + w) : f.m;
  return end - j;
}

// T of the outer block starting at column jo (jbo columns) from its panels' T's.
qdwhp_status build_outer_T(cudaStream_t st, const QRFactors& f, int64_t jo, int jbo, double* G, double* tmp) {
  const int64_t m = f.m, Ro = active_rows(f, jo, jbo);
  const double* Vo = f.Vall + jo + jo * m;
  double* To = f.To + (size_t)(jo / NBO) * NBO * NBO;
  QDWHP_TRY(set_matrix(st, NBO, NBO, 0.0, 0.0, To, NBO));
  if (jbo > NB) QDWHP_TRY(gemm(st, true, false, jbo, jbo, Ro, 1.0, Vo, m, Vo, m, 0.0, G, NBO));
  for (int c0 = 0; c0 < jbo; c0 += NB) {
    const int jb = std::min(NB, jbo - c0);
    const double* Tq = f.T + (size_t)((jo + c0) / NB) * NB * NB;
    QDWHP_TRY(copy_matrix(st, jb, jb, Tq, NB, To + c0 + (size_t)c0 * NBO, NBO));
    if (c0 > 0) {
      QDWHP_TRY(gemm(st, false, false, c0, jb, c0, 1.0, To, NBO, G + (size_t)c0 * NBO, NBO, 0.0, tmp, NBO));
      QDWHP_TRY(gemm(st, false, false, c0, jb, jb, -1.0, tmp, NBO, Tq, NB, 0.0, To + (size_t)c0 * NBO, NBO));
    }
  }
  return QDWHP_OK;
}

}  // namespace

qdwhp_status geqrf(cudaStream_t st, int64_t m, int64_t n, double* A, int64_t lda, QRFactors& f, double* scratch,
                   int64_t band) {
  if (m < n || n < 0 || band < 0 || (band > 0 && band + n != m)) return QDWHP_ERR_ARG;
  // Householder updates C -= V W2 stay native FP64 in every precision mode: V is unit lower
  // trapezoidal and the coefficient columns span many magnitudes, where the emulated
  // product's normwise (row/column-scaled) error is far above FP64's componentwise one.  Only
  // the reduction W = V^T C of the outer blocks follows the caller's precision.
  EmulationScope native_products(nullptr, 0);
  f.m = m;
  f.n = n;
  f.band = band;
  if (n == 0) return QDWHP_OK;
  double* W = scratch;
  double* W2 = W + (size_t)NBO * n;
  const size_t splitk_elems = qr_splitk_elems(n);
  double* splitk = W2 + (size_t)NBO * n;
  double* part = splitk + splitk_elems;
  double* gram = part + 2 * (size_t)kPanelCTAs * kPartStride;
  double* row_slot = gram + (size_t)(kPanelCTAs + 1) * NB * NB;
  double* G = row_slot + 2 * NB;
  double* tmp = G + (size_t)NBO * NBO;
  for (int64_t jo = 0; jo < n; jo += NBO) {
    const int jbo = (int)std::min<int64_t>(NBO, n - jo);
    const int64_t Ro_blk = active_rows(f, jo, jbo);
    for (int64_t j = jo; j < jo + jbo; j += NB) {
      const int jb = (int)std::min<int64_t>(NB, n - j);
      const int64_t R = active_rows(f, j, jb);
      PanelArgs pa;
      pa.R = (int)R;
      pa.jb = jb;
      pa.P = A + j + j * lda;
      pa.lda = lda;
      pa.V = f.Vall + j + j * m;
      pa.ldv = m;
      pa.T = f.T + (size_t)(j / NB) * NB * NB;
      pa.tau = f.tau + j;
      pa.diagR = f.diagR + j;
      pa.part = part;
      pa.gram = gram;
      pa.row_slot = row_slot;
      QDWHP_TRY(launch_panel(st, pa));
      // the outer block's V is zero above each panel's diagonal, and (with a band) below the
      // panel's own rows down to the end of the outer block's rows
      if (j > jo) QDWHP_TRY(set_matrix(st, j - jo, jb, 0.0, 0.0, f.Vall + jo + j * m, m));
      if (jo + Ro_blk > j + R) QDWHP_TRY(set_matrix(st, jo + Ro_blk - (j + R), jb, 0.0, 0.0, f.Vall + (j + R) + j * m, m));
      const int64_t nc = jo + jbo - j - jb;   // the rest of the outer block
      if (nc > 0) {
        double* C = A + j + (j + jb) * lda;
        // W = V^T C ; W2 = T^T W ; C -= V W2
        QDWHP_TRY(gemm(st, true, false, jb, nc, R, 1.0, pa.V, m, C, lda, 0.0, W, jb, FULL, 0.0, splitk,
                       splitk_elems));
        QDWHP_TRY(gemm(st, true, false, jb, nc, jb, 1.0, pa.T, NB, W, jb, 0.0, W2, jb));
        QDWHP_TRY(gemm(st, false, false, R, nc, jb, -1.0, pa.V, m, W2, jb, 1.0, C, lda));
      }
    }
    QDWHP_TRY(build_outer_T(st, f, jo, jbo, G, tmp));
    const int64_t nc = n - jo - jbo;   // trailing columns: one update with the outer block
    if (nc > 0) {
      const int64_t Ro = Ro_blk;
      const double* Vo = f.Vall + jo + jo * m;
      const double* To = f.To + (size_t)(jo / NBO) * NBO * NBO;
      double* C = A + jo + (jo + jbo) * lda;
      {
        // the reduction W = V^T C (rows of V^T: whole reflectors) may use the caller's emulation
        EmulationScope reduction(native_products.prev_ws, native_products.prev_bytes);
        QDWHP_TRY(gemm(st, true, false, jbo, nc, Ro, 1.0, Vo, m, C, lda, 0.0, W, jbo, FULL, 0.0, splitk,
                       splitk_elems));
      }
      QDWHP_TRY(gemm(st, true, false, jbo, nc, jbo, 1.0, To, NBO, W, jbo, 0.0, W2, jbo));
      QDWHP_TRY(gemm(st, false, false, Ro, nc, jbo, -1.0, Vo, m, W2, jbo, 1.0, C, lda));
    }
  }
  return QDWHP_OK;
}

namespace {

// C(jo:, :) -= V_o (T_o (V_o^T C(jo:, :))) for the outer blocks from the one holding panel
// block last_block down to 0, i.e. C := Q C restricted to those reflectors (the extra panels of
// the last outer block act on rows that are zero in the orgqr use and belong to Q otherwise).
qdwhp_status apply_blocks(cudaStream_t st, const QRFactors& f, int64_t last_block, double* C, int64_t ncols,
                          int64_t ldc, double* scratch) {
  EmulationScope native_products(nullptr, 0);   // as in geqrf
  const int64_t m = f.m, n = f.n;
  double* W = scratch;
  double* W2 = W + (size_t)NBO * ncols;
  const size_t splitk_elems = qr_splitk_elems(ncols);
  double* splitk = W2 + (size_t)NBO * ncols;
  for (int64_t po = (last_block * NB) / NBO; po >= 0; --po) {
    const int64_t jo = po * NBO;
    const int jbo = (int)std::min<int64_t>(NBO, n - jo);
    const int64_t Ro = active_rows(f, jo, jbo);
    const double* Vo = f.Vall + jo + jo * m;
    const double* To = f.To + (size_t)po * NBO * NBO;
    double* Cj = C + jo;
    {
      EmulationScope reduction(native_products.prev_ws, native_products.prev_bytes);   // as in geqrf
      QDWHP_TRY(gemm(st, true, false, jbo, ncols, Ro, 1.0, Vo, m, Cj, ldc, 0.0, W, jbo, FULL, 0.0, splitk,
                     splitk_elems));
    }
    QDWHP_TRY(gemm(st, false, false, jbo, ncols, jbo, 1.0, To, NBO, W, jbo, 0.0, W2, jbo));
    QDWHP_TRY(gemm(st, false, false, Ro, ncols, jbo, -1.0, Vo, m, W2, jbo, 1.0, Cj, ldc));
  }
  return QDWHP_OK;
}

}  // namespace

qdwhp_status orgqr_columns(cudaStream_t st, const QRFactors& f, int64_t col0, int64_t ncols, double* C, int64_t ldc,
                           double* scratch) {
  const int64_t m = f.m, n = f.n;
  if (col0 < 0 || ncols < 0 || col0 + ncols > n) return QDWHP_ERR_ARG;
  if (ncols == 0) return QDWHP_OK;
  QDWHP_TRY(set_matrix(st, m, ncols, 0.0, 0.0, C, ldc));
  QDWHP_TRY(set_matrix(st, ncols, ncols, 0.0, 1.0, C + col0, ldc));
  // Blocks whose first column is past the selected range act on zero rows: skip them.
  return apply_blocks(st, f, (col0 + ncols - 1) / NB, C, ncols, ldc, scratch);
}

qdwhp_status ormqr_left(cudaStream_t st, const QRFactors& f, double* C, int64_t ncols, int64_t ldc, double* scratch) {
  if (ncols <= 0 || f.n <= 0) return QDWHP_OK;
  return apply_blocks(st, f, (f.n - 1) / NB, C, ncols, ldc, scratch);
}

}  // namespace qdwhp
