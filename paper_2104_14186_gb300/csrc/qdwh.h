// Internal interfaces of qdwh.cu (QDWH steps and the device weight schedule).
#pragma once

#include "internal.h"

namespace qdwhp {

constexpr int kMaxSteps = 12;
constexpr int kZoloMaxR = 8;

struct Schedule {
  double ell0;
  double abc[3 * kMaxSteps];
  double ell_after[kMaxSteps];
  int use_qr[kMaxSteps];
  int nsteps;
};

// Zolo-PD: per iteration the type (2r+1, 2r) Zolotarev function on [ell_k, 1],
// Z(x) = mhat x (1 + sum_j a_j / (x^2 + c_{2j-1})), and which terms use the QR form.
struct ZoloSchedule {
  double ell0;
  int r;
  int nsteps;
  double c[kMaxSteps][2 * kZoloMaxR];   // c_1 .. c_2r
  double a[kMaxSteps][kZoloMaxR];
  double mhat[kMaxSteps];
  double ell_after[kMaxSteps];
  int use_qr[kMaxSteps][kZoloMaxR];
};

struct QdwhWs {
  int64_t m = 0, n = 0;
  double* Z = nullptr;        // n x n: Z, then its Cholesky factor L (lower)
  double* Linv = nullptr;     // inverses of the diagonal leaves of L
  double* Y = nullptr;        // m x n solve / product buffer
  double* scratch = nullptr;
  int* fail = nullptr;        // first failing Cholesky column (0 = none), reset by the caller
  double* diff_parts = nullptr;
  double* diff = nullptr;     // ||X_k - X_{k-1}||_F^2 per step
  bool has_qr = false;
  double* S = nullptr;        // (m+n) x n stacked matrix, then its explicit Q
  QRFactors qf;
  double* qr_scratch = nullptr;
  // FP32 buffers of the reduced-precision Cholesky steps (QDWHP_MIXED)
  bool has_f32 = false;
  float* X32 = nullptr;       // m x n
  float* Z32 = nullptr;       // n x n
  float* Linv32 = nullptr;
  float* Y32 = nullptr;       // m x n
  float* scratch32 = nullptr;
  // Zolo-PD buffers
  bool has_zolo = false;
  double* G = nullptr;        // n x n Gram matrix X^T X (lower)
  double* Acc = nullptr;      // m x n sum of the terms
};

void carve_qdwh(Arena& ar, int64_t m, int64_t n, bool need_qr, QdwhWs& w, bool need_f32 = false,
                bool need_zolo = false);
// Weights from ell_0 (device scalar if ell0_dev != null, else ell0_host); fixed_iters > 0
// runs exactly that many steps, otherwise until |ell - 1| < 5 eps.
qdwhp_status dwh_schedule(cudaStream_t st, const double* ell0_dev, double ell0_host, int fixed_iters, double c_qr,
                          Schedule* out_dev);
qdwhp_status chol_step(cudaStream_t st, int64_t m, int64_t n, double* X, int64_t ldx, double a, double b, double c,
                       QdwhWs& w, int step);
qdwhp_status qr_step(cudaStream_t st, int64_t m, int64_t n, double* X, int64_t ldx, double a, double b, double c,
                     QdwhWs& w, int step);
// Cholesky-based step in FP32 on w.X32 (m x n, ld m) with FP32 products, factorisation and solves.
qdwhp_status chol_step_f32(cudaStream_t st, int64_t m, int64_t n, double a, double b, double c, QdwhWs& w, int step);
// Zolo-PD schedule from ell0 (host value) with r terms per iteration until |ell - 1| < 5 eps;
// a term takes the QR form when 1 / c_{2j-1} > c_qr.
qdwhp_status zolo_schedule(cudaStream_t st, double ell0, int r, double c_qr, ZoloSchedule* out_dev);
// Runs the Zolo-PD iterations on X (FP64; w needs has_qr and has_zolo).  Counts the terms
// formed by QR and by Cholesky.
qdwhp_status run_zolo(cudaStream_t st, int64_t m, int64_t n, double* X, int64_t ldx, const ZoloSchedule& z,
                      QdwhWs& w, int* n_qr_terms, int* n_chol_terms);
// Runs the schedule's steps on X (FP64): QR-based steps in FP64; with `mixed`, every Cholesky-based
// step but the last in FP32 (X converted down before and back up after), the last in FP64.
// Returns the number of FP32 steps in *n_f32.
qdwhp_status run_schedule(cudaStream_t st, int64_t m, int64_t n, double* X, int64_t ldx, const Schedule& sched,
                          bool mixed, QdwhWs& w, int* n_qr, int* n_chol, int* n_f32);

}  // namespace qdwhp
