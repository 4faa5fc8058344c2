// QDWH iteration (Section 3.1): dynamical weights on the device and the two
// practical step forms.
//   Cholesky-based (eq. practical-polar-chol):
//     Z = I + c X^T X (lower SYRK with the identity folded into the epilogue),
//     L = chol(Z) (W = L^T), Y = (X L^{-T}) L^{-1} = X W^{-1} W^{-T},
//     X <- (b/c) X + (a - b/c) Y.
//   QR-based (eq. practical-polar-qr):
//     [sqrt(c) X; I] = [Q1; Q2] R,  X <- (b/c) X + (1/sqrt(c)) (a - b/c) Q1 Q2^T.
// Each step also reports ||X_k - X_{k-1}||_F (the Section 5 listing's diagnostic).
//
// Zolo-PD (the higher-order Zolotarev variant that Section 3.1 sets beside QDWH and the
// conclusion leaves as future work; Nakatsukasa and Freund, SIAM Review 2016): iteration k
// applies the best type (2r+1, 2r) rational approximation of sign on [ell_k, 1],
//     X <- mhat (X + sum_j a_j X (X^T X + c_{2j-1} I)^{-1}),
// with c_i = ell^2 sc^2(i K' / (2r+1); ell'), ell' = sqrt(1 - ell^2), K' = K(ell'), the
// partial-fraction weights a_j and mhat normalising Z(1) = 1; ell_{k+1} = Z(ell_k).  One
// Gram matrix X^T X serves every Cholesky-formed term; a term whose shift is small
// (1 / c_{2j-1} > c_qr) is formed from [X; sqrt(c) I] = [Q1; Q2] R as Q1 Q2^T / sqrt(c).
// r = 1 is the QDWH step.
#include "internal.h"
#include "qdwh.h"

namespace qdwhp {

namespace {

// Weights of every step from ell_0 (Section 3.1 and the weight lines of the Section 5
// listing): L2 = l^2, d = cbrt(4(1 - L2)/L2^2), a = sqrt(1+d) + sqrt(8 - 4d + 8(2 - L2)/(L2 sqrt(1+d)))/2,
// b = (a-1)^2/4, c = a + b - 1, l <- l (a + b L2)/(1 + c L2).  Stops when |l - 1| < 5 * 2^-52
// or after fixed_iters steps when fixed_iters > 0.
__global__ void dwh_schedule_kernel(const double* ell0_dev, double ell0_host, int fixed_iters, double c_qr,
                                    Schedule* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double ell = ell0_dev ? *ell0_dev : ell0_host;
  out->ell0 = ell;
  int n = 0;
  while (n < kMaxSteps) {
    if (fixed_iters > 0) {
      if (n >= fixed_iters) break;
    } else if (fabs(ell - 1.0) < 5.0 * 0x1.0p-52) {
      break;
    }
    double a, b, c, nxt;
    if (ell >= 1.0) {
      a = 3.0;
      b = 1.0;
      c = 3.0;
      nxt = 1.0;
    } else {
      const double L2 = ell * ell;
      const double d = cbrt(4.0 * (1.0 - L2) / (L2 * L2));
      const double sqd = sqrt(1.0 + d);
      a = sqd + 0.5 * sqrt(8.0 - 4.0 * d + 8.0 * (2.0 - L2) / (L2 * sqd));
      b = (a - 1.0) * (a - 1.0) / 4.0;
      c = a + b - 1.0;
      nxt = fmin(ell * (a + b * L2) / (1.0 + c * L2), 1.0);
    }
    out->abc[3 * n + 0] = a;
    out->abc[3 * n + 1] = b;
    out->abc[3 * n + 2] = c;
    out->ell_after[n] = nxt;
    out->use_qr[n] = (c > c_qr) ? 1 : 0;
    ell = nxt;
    ++n;
  }
  out->nsteps = n;
}

// Jacobi elliptic sn(u) and cn(u) of modulus k = sqrt(1 - kc^2), given the complementary
// modulus kc, for 0 <= u <= K(k) / 2, by Landen's descending transformation (DLMF 22.7.1-3):
// with k1 = (1 - kc) / (1 + kc) and v = u / (1 + k1),
//   sn(u, k) = (1 + k1) sn(v, k1) / D,  cn(u, k) = cn(v, k1) dn(v, k1) / D,
//   dn(u, k) = (1 - k1 sn^2(v, k1)) / D,  D = 1 + k1 sn^2(v, k1),
// repeated until the modulus is below 2^-27, where sn, cn, dn are sin, cos, 1 to rounding.
// Every quantity is carried through its complement: 1 - k1 = 2 kc / (1 + kc),
// kc1 = 2 sqrt(kc) / (1 + kc), and dn's numerator is (1 - k1) + k1 cn^2, so nothing cancels
// when k is within rounding of 1.  Since u <= K / 2 ends at an argument <= pi / 4, cn stays
// well away from 0 at the bottom, and all steps multiply or divide positive numbers: sn and
// cn keep a relative accuracy of a few ulps for any kc in (0, 1].
__device__ void elliptic_sn_cn(double u, double kc, double* sn_out, double* cn_out) {
  constexpr int kLandenMax = 40;
  double k[kLandenMax], omk[kLandenMax];
  int levels = 0;
  double v = u;
  while (levels < kLandenMax) {
    const double k1 = (1.0 - kc) / (1.0 + kc);
    k[levels] = k1;
    omk[levels] = 2.0 * kc / (1.0 + kc);
    ++levels;
    kc = 2.0 * sqrt(kc) / (1.0 + kc);
    v /= 1.0 + k1;
    if (k1 < 0x1.0p-27) break;
  }
  double sn = sin(v), cn = cos(v), dn = 1.0;
  for (int i = levels - 1; i >= 0; --i) {
    const double den = 1.0 + k[i] * sn * sn;
    const double sn_up = (1.0 + k[i]) * sn / den;
    const double cn_up = cn * dn / den;
    dn = (omk[i] + k[i] * cn * cn) / den;
    sn = sn_up;
    cn = cn_up;
  }
  *sn_out = sn;
  *cn_out = cn;
}

// Complete elliptic integral of the first kind K of the modulus whose complement is kc:
// K = pi / (2 AGM(1, kc)).
__device__ double elliptic_k_of_complement(double kc) {
  double a = 1.0, b = kc;
  for (int i = 0; i < 64 && fabs(a - b) > 0x1.0p-53 * a; ++i) {
    const double an = 0.5 * (a + b);
    b = sqrt(a * b);
    a = an;
  }
  return 3.14159265358979323846 / (2.0 * a);
}

__global__ void zolo_schedule_kernel(double ell0, int r, double c_qr, ZoloSchedule* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double ell = ell0;
  out->ell0 = ell0;
  out->r = r;
  int n = 0;
  while (n < kMaxSteps && ell < 1.0 && fabs(ell - 1.0) >= 5.0 * 0x1.0p-52) {
    // K' = K(ell'), whose complementary modulus is ell; c_i = ell^2 sc^2(i K' / (2r+1); ell').
    // Past K'/2, sc(K' - v) = cn(v) / (ell sn(v)) keeps cn away from 0: c_i = cs^2(v).
    const double Kp = elliptic_k_of_complement(ell);
    const int d = 2 * r + 1;
    double* c = out->c[n];
    for (int i = 1; i <= 2 * r; ++i) {
      double sn, cn;
      if (2 * i <= d) {
        elliptic_sn_cn(i * Kp / d, ell, &sn, &cn);
        c[i - 1] = ell * ell * (sn / cn) * (sn / cn);
      } else {
        elliptic_sn_cn((d - i) * Kp / d, ell, &sn, &cn);
        c[i - 1] = (cn / sn) * (cn / sn);
      }
    }
    double mhat = 1.0, zl = ell;
    for (int j = 0; j < r; ++j) {
      const double codd = c[2 * j];
      double num = 1.0, den = 1.0;
      for (int k = 0; k < r; ++k) {
        num *= codd - c[2 * k + 1];
        if (k != j) den *= codd - c[2 * k];
      }
      out->a[n][j] = -num / den;
      out->use_qr[n][j] = (1.0 / codd > c_qr) ? 1 : 0;
      mhat *= (1.0 + codd) / (1.0 + c[2 * j + 1]);
      zl *= (ell * ell + c[2 * j + 1]) / (ell * ell + codd);
    }
    out->mhat[n] = mhat;
    const double nxt = fmin(mhat * zl, 1.0);
    out->ell_after[n] = nxt;
    ell = nxt;
    ++n;
  }
  out->nsteps = n;
}

}  // namespace

qdwhp_status zolo_schedule(cudaStream_t st, double ell0, int r, double c_qr, ZoloSchedule* out_dev) {
  if (r < 1 || r > kZoloMaxR || !(ell0 > 0.0)) return QDWHP_ERR_ARG;
  zolo_schedule_kernel<<<1, 32, 0, st>>>(ell0, r, c_qr, out_dev);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status dwh_schedule(cudaStream_t st, const double* ell0_dev, double ell0_host, int fixed_iters, double c_qr,
                          Schedule* out_dev) {
  dwh_schedule_kernel<<<1, 32, 0, st>>>(ell0_dev, ell0_host, fixed_iters, c_qr, out_dev);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

void carve_qdwh(Arena& ar, int64_t m, int64_t n, bool need_qr, QdwhWs& w, bool need_f32, bool need_zolo) {
  w.m = m;
  w.n = n;
  w.Z = ar.take<double>((size_t)n * n);
  w.Linv = ar.take<double>(potrf_linv_elems(n));
  w.Y = ar.take<double>((size_t)m * n);
  w.scratch = ar.take<double>(std::max(potrf_scratch_elems(n), trsm_scratch_elems(m, n)));
  w.fail = ar.take<int>(4);
  w.diff_parts = ar.take<double>(kDiffParts);
  w.diff = ar.take<double>(kMaxSteps);
  w.has_qr = need_qr;
  if (need_qr) {
    const int64_t mm = m + n;
    w.S = ar.take<double>((size_t)mm * n);
    w.qf.Vall = ar.take<double>((size_t)mm * n);
    w.qf.T = ar.take<double>((size_t)ceil_div(n, kQRNB) * kQRNB * kQRNB);
    w.qf.To = ar.take<double>(qr_to_elems(n));
    w.qf.tau = ar.take<double>(n);
    w.qf.diagR = ar.take<double>(n);
    w.qr_scratch = ar.take<double>(qr_scratch_elems(mm, n));
  }
  w.has_zolo = need_zolo;
  if (need_zolo) {
    w.G = ar.take<double>((size_t)n * n);
    w.Acc = ar.take<double>((size_t)m * n);
  }
  w.has_f32 = need_f32;
  if (need_f32) {
    w.X32 = ar.take<float>((size_t)m * n);
    w.Z32 = ar.take<float>((size_t)n * n);
    w.Linv32 = ar.take<float>(potrf_linv_elems(n));
    w.Y32 = ar.take<float>((size_t)m * n);
    w.scratch32 = ar.take<float>(std::max(potrf_scratch_elems(n), trsm_scratch_elems(m, n)));
  }
}

qdwhp_status chol_step(cudaStream_t st, int64_t m, int64_t n, double* X, int64_t ldx, double a, double b, double c,
                       QdwhWs& w, int step) {
  // Z = I + c X^T X (lower)
  QDWHP_TRY(gemm(st, true, false, n, n, m, c, X, ldx, X, ldx, 0.0, w.Z, n, LOWER, 1.0));
  QDWHP_TRY(potrf(st, n, w.Z, n, w.Linv, w.scratch, w.fail));
  QDWHP_TRY(copy_matrix(st, m, n, X, ldx, w.Y, m));
  QDWHP_TRY(trsm_right_lower(st, true, m, n, w.Y, m, w.Z, n, w.Linv, w.scratch));    // X W^{-1}
  QDWHP_TRY(trsm_right_lower(st, false, m, n, w.Y, m, w.Z, n, w.Linv, w.scratch));   // (X W^{-1}) W^{-T}
  QDWHP_TRY(axpby_diff(st, m, n, b / c, X, ldx, a - b / c, w.Y, m, w.diff_parts));
  return reduce_parts(st, w.diff_parts, kDiffParts, w.diff + step);
}

qdwhp_status qr_step(cudaStream_t st, int64_t m, int64_t n, double* X, int64_t ldx, double a, double b, double c,
                     QdwhWs& w, int step) {
  if (!w.has_qr) return QDWHP_ERR_ARG;
  const int64_t mm = m + n;
  const double sc = sqrt(c);
  // S = [sqrt(c) X; I]
  QDWHP_TRY(axpby(st, m, n, sc, X, ldx, 0.0, w.S, mm));
  QDWHP_TRY(set_matrix(st, n, n, 0.0, 1.0, w.S + m, mm));
  QDWHP_TRY(geqrf(st, mm, n, w.S, mm, w.qf, w.qr_scratch, m));   // the identity block's zeros are skipped
  // explicit [Q1; Q2] (the compact factors live in qf, so S can be overwritten)
  QDWHP_TRY(orgqr_columns(st, w.qf, 0, n, w.S, mm, w.qr_scratch));
  // Y = Q1 Q2^T
  QDWHP_TRY(gemm(st, false, true, m, n, n, 1.0, w.S, mm, w.S + m, mm, 0.0, w.Y, m));
  QDWHP_TRY(axpby_diff(st, m, n, b / c, X, ldx, (a - b / c) / sc, w.Y, m, w.diff_parts));
  return reduce_parts(st, w.diff_parts, kDiffParts, w.diff + step);
}

// One Zolo-PD iteration (see the file header).
qdwhp_status zolo_step(cudaStream_t st, int64_t m, int64_t n, double* X, int64_t ldx, const ZoloSchedule& z,
                       int step, QdwhWs& w, int* n_qr_terms, int* n_chol_terms) {
  if (!w.has_zolo || !w.has_qr) return QDWHP_ERR_ARG;
  const int r = z.r;
  const int64_t mm = m + n;
  bool any_chol = false;
  for (int j = 0; j < r; ++j) any_chol |= !z.use_qr[step][j];
  // G = X^T X (lower; the upper triangle held at 0 so that G + c I copies finite values),
  // shared by the Cholesky-formed terms
  if (any_chol) {
    QDWHP_TRY(set_matrix(st, n, n, 0.0, 0.0, w.G, n));
    QDWHP_TRY(gemm(st, true, false, n, n, m, 1.0, X, ldx, X, ldx, 0.0, w.G, n, LOWER));
  }
  QDWHP_TRY(copy_matrix(st, m, n, X, ldx, w.Acc, m));
  for (int j = 0; j < r; ++j) {
    const double cj = z.c[step][2 * j], aj = z.a[step][j];
    if (z.use_qr[step][j]) {
      // [X; sqrt(c) I] = [Q1; Q2] R:  X (X^T X + c I)^{-1} = Q1 Q2^T / sqrt(c)
      const double sc = sqrt(cj);
      QDWHP_TRY(copy_matrix(st, m, n, X, ldx, w.S, mm));
      QDWHP_TRY(set_matrix(st, n, n, 0.0, sc, w.S + m, mm));
      QDWHP_TRY(geqrf(st, mm, n, w.S, mm, w.qf, w.qr_scratch, m));
      QDWHP_TRY(orgqr_columns(st, w.qf, 0, n, w.S, mm, w.qr_scratch));
      QDWHP_TRY(gemm(st, false, true, m, n, n, aj / sc, w.S, mm, w.S + m, mm, 1.0, w.Acc, m));
      ++*n_qr_terms;
    } else {
      // G + c I = L L^T:  X (G + c I)^{-1} = (X L^{-T}) L^{-1}
      QDWHP_TRY(axpby(st, n, n, 1.0, w.G, n, 0.0, w.Z, n, cj));
      QDWHP_TRY(potrf(st, n, w.Z, n, w.Linv, w.scratch, w.fail));
      QDWHP_TRY(copy_matrix(st, m, n, X, ldx, w.Y, m));
      QDWHP_TRY(trsm_right_lower(st, true, m, n, w.Y, m, w.Z, n, w.Linv, w.scratch));
      QDWHP_TRY(trsm_right_lower(st, false, m, n, w.Y, m, w.Z, n, w.Linv, w.scratch));
      QDWHP_TRY(axpby(st, m, n, aj, w.Y, m, 1.0, w.Acc, m));
      ++*n_chol_terms;
    }
  }
  // X <- mhat Acc, with ||X_new - X_old||_F^2
  QDWHP_TRY(axpby_diff(st, m, n, 0.0, X, ldx, z.mhat[step], w.Acc, m, w.diff_parts));
  return reduce_parts(st, w.diff_parts, kDiffParts, w.diff + step);
}

qdwhp_status run_zolo(cudaStream_t st, int64_t m, int64_t n, double* X, int64_t ldx, const ZoloSchedule& z,
                      QdwhWs& w, int* n_qr_terms, int* n_chol_terms) {
  *n_qr_terms = *n_chol_terms = 0;
  for (int i = 0; i < z.nsteps; ++i) QDWHP_TRY(zolo_step(st, m, n, X, ldx, z, i, w, n_qr_terms, n_chol_terms));
  return QDWHP_OK;
}

qdwhp_status chol_step_f32(cudaStream_t st, int64_t m, int64_t n, double a, double b, double c, QdwhWs& w,
                           int step) {
  if (!w.has_f32) return QDWHP_ERR_ARG;
  QDWHP_TRY(gemm(st, true, false, n, n, m, (float)c, w.X32, m, w.X32, m, 0.0f, w.Z32, n, LOWER, 1.0f));
  QDWHP_TRY(potrf(st, n, w.Z32, n, w.Linv32, w.scratch32, w.fail));
  QDWHP_TRY(copy_matrix(st, m, n, w.X32, m, w.Y32, m));
  QDWHP_TRY(trsm_right_lower(st, true, m, n, w.Y32, m, w.Z32, n, w.Linv32, w.scratch32));
  QDWHP_TRY(trsm_right_lower(st, false, m, n, w.Y32, m, w.Z32, n, w.Linv32, w.scratch32));
  QDWHP_TRY(axpby_diff(st, m, n, (float)(b / c), w.X32, m, (float)(a - b / c), w.Y32, m, w.diff_parts));
  return reduce_parts(st, w.diff_parts, kDiffParts, w.diff + step);
}

qdwhp_status run_schedule(cudaStream_t st, int64_t m, int64_t n, double* X, int64_t ldx, const Schedule& sched,
                          bool mixed, QdwhWs& w, int* n_qr, int* n_chol, int* n_f32) {
  *n_qr = *n_chol = *n_f32 = 0;
  int last_chol = -1;
  for (int i = 0; i < sched.nsteps; ++i)
    if (!sched.use_qr[i]) last_chol = i;
  bool in_f32 = false;
  for (int i = 0; i < sched.nsteps; ++i) {
    const double a = sched.abc[3 * i], b = sched.abc[3 * i + 1], c = sched.abc[3 * i + 2];
    const bool low = mixed && !sched.use_qr[i] && i != last_chol;
    if (low && !in_f32) {
      QDWHP_TRY(convert(st, m, n, X, ldx, w.X32, m));
      in_f32 = true;
    } else if (!low && in_f32) {
      QDWHP_TRY(convert(st, m, n, w.X32, m, X, ldx));
      in_f32 = false;
    }
    if (sched.use_qr[i]) {
      QDWHP_TRY(qr_step(st, m, n, X, ldx, a, b, c, w, i));
      ++*n_qr;
    } else if (low) {
      QDWHP_TRY(chol_step_f32(st, m, n, a, b, c, w, i));
      ++*n_chol;
      ++*n_f32;
    } else {
      QDWHP_TRY(chol_step(st, m, n, X, ldx, a, b, c, w, i));
      ++*n_chol;
    }
  }
  if (in_f32) QDWHP_TRY(convert(st, m, n, w.X32, m, X, ldx));
  return QDWHP_OK;
}

}  // namespace qdwhp

// ---------------------------------------------------------------------------------------
// C-ABI building blocks.

using namespace qdwhp;

extern "C" {

QDWHP_API qdwhp_status qdwhp_gemm_f64(int transa, int transb, int64_t m, int64_t n, int64_t k, double alpha,
                                      const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                                      double* C, int64_t ldc, void* stream) {
  if (m < 0 || n < 0 || k < 0) return QDWHP_ERR_ARG;
  if (m == 0 || n == 0) return QDWHP_OK;
  const int64_t rowsA = transa ? k : m, rowsB = transb ? n : k;
  if (C == nullptr || ldc < m || lda < std::max<int64_t>(1, rowsA) || ldb < std::max<int64_t>(1, rowsB))
    return QDWHP_ERR_ARG;
  if (k > 0 && (A == nullptr || B == nullptr)) return QDWHP_ERR_ARG;
  return gemm((cudaStream_t)stream, transa != 0, transb != 0, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

QDWHP_API size_t qdwhp_gemm_f64_emulated_workspace_bytes(int64_t m, int64_t n, int64_t k) {
  return gemm_ozaki_ws_bytes(m, n, k);
}

QDWHP_API qdwhp_status qdwhp_gemm_f64_emulated(int transa, int transb, int64_t m, int64_t n, int64_t k,
                                               double alpha, const double* A, int64_t lda, const double* B,
                                               int64_t ldb, double beta, double* C, int64_t ldc, void* workspace,
                                               size_t ws_bytes, void* stream) {
  if (m < 0 || n < 0 || k < 0) return QDWHP_ERR_ARG;
  if (m == 0 || n == 0) return QDWHP_OK;
  const int64_t rowsA = transa ? k : m, rowsB = transb ? n : k;
  if (C == nullptr || ldc < m || lda < std::max<int64_t>(1, rowsA) || ldb < std::max<int64_t>(1, rowsB))
    return QDWHP_ERR_ARG;
  if (k > 0 && (A == nullptr || B == nullptr)) return QDWHP_ERR_ARG;
  if (k > 0 && (workspace == nullptr || ((uintptr_t)workspace & 15) != 0)) return QDWHP_ERR_ARG;
  return gemm_ozaki((cudaStream_t)stream, transa != 0, transb != 0, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                    FULL, 0.0, workspace, ws_bytes);
}

QDWHP_API size_t qdwhp_gemm_f32_bf16x6_workspace_bytes(int64_t m, int64_t n, int64_t k) {
  return gemm_bf16x6_ws_bytes(m, n, k);
}

QDWHP_API qdwhp_status qdwhp_gemm_f32_bf16x6(int transa, int transb, int64_t m, int64_t n, int64_t k, float alpha,
                                             const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                                             float* C, int64_t ldc, void* workspace, size_t ws_bytes, void* stream) {
  if (m < 0 || n < 0 || k < 0) return QDWHP_ERR_ARG;
  if (m == 0 || n == 0) return QDWHP_OK;
  const int64_t rowsA = transa ? k : m, rowsB = transb ? n : k;
  if (C == nullptr || ldc < m || lda < std::max<int64_t>(1, rowsA) || ldb < std::max<int64_t>(1, rowsB))
    return QDWHP_ERR_ARG;
  if (k > 0 && (A == nullptr || B == nullptr)) return QDWHP_ERR_ARG;
  if (k > 0 && (workspace == nullptr || ((uintptr_t)workspace & 15) != 0)) return QDWHP_ERR_ARG;
  return gemm_bf16x6((cudaStream_t)stream, transa != 0, transb != 0, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                     FULL, 0.0f, workspace, ws_bytes);
}

QDWHP_API size_t qdwhp_potrf_workspace_bytes(int64_t n) {
  Arena ar;
  ar.dry = true;
  ar.take<double>(potrf_linv_elems(n));
  ar.take<double>(potrf_scratch_elems(n));
  ar.take<int>(4);
  return ar.used;
}

QDWHP_API qdwhp_status qdwhp_potrf_f64(int64_t n, double* Z, int64_t ldz, void* workspace, size_t ws_bytes,
                                       int* info_host, void* stream) {
  if (n < 0 || (n > 0 && (Z == nullptr || ldz < n))) return QDWHP_ERR_ARG;
  if (info_host) *info_host = 0;
  if (n == 0) return QDWHP_OK;
  if (workspace == nullptr || ws_bytes < qdwhp_potrf_workspace_bytes(n)) return QDWHP_ERR_NOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar{(char*)workspace, ws_bytes};
  double* Linv = ar.take<double>(potrf_linv_elems(n));
  double* scratch = ar.take<double>(potrf_scratch_elems(n));
  int* fail = ar.take<int>(4);
  QDWHP_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int), st));
  QDWHP_TRY(potrf(st, n, Z, ldz, Linv, scratch, fail));
  int h = 0;
  QDWHP_CUDA_TRY(cudaMemcpyAsync(&h, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
  QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  if (info_host) *info_host = h;
  return h ? QDWHP_ERR_BREAKDOWN : QDWHP_OK;
}

QDWHP_API size_t qdwhp_qr_workspace_bytes(int64_t m, int64_t n) {
  Arena ar;
  ar.dry = true;
  ar.take<double>((size_t)m * n);
  ar.take<double>((size_t)ceil_div(std::max<int64_t>(n, 1), kQRNB) * kQRNB * kQRNB);
  ar.take<double>(qr_to_elems(n));
  ar.take<double>(n);
  ar.take<double>(n);
  ar.take<double>(qr_scratch_elems(m, n));
  return ar.used;
}

QDWHP_API qdwhp_status qdwhp_qr_f64(int64_t m, int64_t n, double* A, int64_t lda, double* Q, int64_t ldq, double* R,
                                    int64_t ldr, void* workspace, size_t ws_bytes, void* stream) {
  if (m < n || n < 0) return QDWHP_ERR_ARG;
  if (n == 0) return QDWHP_OK;
  if (!A || !Q || !R || lda < m || ldq < m || ldr < n) return QDWHP_ERR_ARG;
  if (workspace == nullptr || ws_bytes < qdwhp_qr_workspace_bytes(m, n)) return QDWHP_ERR_NOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar{(char*)workspace, ws_bytes};
  QRFactors f;
  f.Vall = ar.take<double>((size_t)m * n);
  f.T = ar.take<double>((size_t)ceil_div(n, kQRNB) * kQRNB * kQRNB);
  f.To = ar.take<double>(qr_to_elems(n));
  f.tau = ar.take<double>(n);
  f.diagR = ar.take<double>(n);
  double* scratch = ar.take<double>(qr_scratch_elems(m, n));
  QDWHP_TRY(geqrf(st, m, n, A, lda, f, scratch));
  QDWHP_TRY(copy_upper(st, n, A, lda, R, ldr));
  return orgqr_columns(st, f, 0, n, Q, ldq, scratch);
}

QDWHP_API size_t qdwhp_qdwh_workspace_bytes(int64_t m, int64_t n) {
  Arena ar;
  ar.dry = true;
  QdwhWs w;
  carve_qdwh(ar, m, n, true, w);
  return ar.used;
}

QDWHP_API qdwhp_status qdwhp_qdwh_steps_f64(int64_t m, int64_t n, double* X, int64_t ldx, int32_t nsteps,
                                            const double* abc_host, const int32_t* use_qr_host, double* conv_host,
                                            void* workspace, size_t ws_bytes, void* stream) {
  if (m < n || n < 1 || X == nullptr || ldx < m || nsteps < 0 || nsteps > kMaxSteps) return QDWHP_ERR_ARG;
  if (nsteps > 0 && (abc_host == nullptr || use_qr_host == nullptr)) return QDWHP_ERR_ARG;
  if (workspace == nullptr || ws_bytes < qdwhp_qdwh_workspace_bytes(m, n)) return QDWHP_ERR_NOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar{(char*)workspace, ws_bytes};
  QdwhWs w;
  carve_qdwh(ar, m, n, true, w);
  QDWHP_CUDA_TRY(cudaMemsetAsync(w.fail, 0, sizeof(int), st));
  for (int i = 0; i < nsteps; ++i) {
    const double a = abc_host[3 * i], b = abc_host[3 * i + 1], c = abc_host[3 * i + 2];
    if (use_qr_host[i])
      QDWHP_TRY(qr_step(st, m, n, X, ldx, a, b, c, w, i));
    else
      QDWHP_TRY(chol_step(st, m, n, X, ldx, a, b, c, w, i));
  }
  double diffs[kMaxSteps];
  int fail = 0;
  if (nsteps > 0) QDWHP_CUDA_TRY(cudaMemcpyAsync(diffs, w.diff, sizeof(double) * nsteps, cudaMemcpyDeviceToHost, st));
  QDWHP_CUDA_TRY(cudaMemcpyAsync(&fail, w.fail, sizeof(int), cudaMemcpyDeviceToHost, st));
  QDWHP_CUDA_TRY(cudaStreamSynchronize(st));
  if (conv_host)
    for (int i = 0; i < nsteps; ++i) conv_host[i] = sqrt(diffs[i]);
  return fail ? QDWHP_ERR_BREAKDOWN : QDWHP_OK;
}

}  // extern "C"
