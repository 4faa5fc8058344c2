/*
 * qdwhp: partial symmetric eigensolver and partial SVD by dynamically weighted
 * Halley (QDWH) iterations, for one NVIDIA GB300 (sm_103a).
 *
 * Method: Keyes, Ltaief, Nakatsukasa, Sukkari, "High-Performance Partial Spectrum
 * Computation for Symmetric eigenvalue problems and the SVD" (arXiv 2104.14186):
 * Algorithm 1 (QDWHpartial-EIG), Algorithm 2 (QDWHpartial-SVD), the QDWH steps of
 * Section 3.1 (eqs. practical-polar-qr and practical-polar-chol) and the index rule
 * of Section 4.1.
 *
 * Conventions for every entry point below:
 *   - Matrices are FP64, column-major, with a leading dimension >= the row count.
 *   - Matrix and vector arguments are DEVICE pointers unless the name ends in
 *     `_host`; the caller owns all memory and the library frees nothing it did
 *     not allocate (it allocates nothing: scratch comes from `workspace`).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; entry points that need a scalar from the device
 *     (subspace size, thresholds) synchronise that stream before they return.
 *   - A non-OK status leaves the outputs undefined.  No call falls back to the CPU.
 *   - Errors: QDWHP_ERR_ARG for bad sizes/pointers (nothing is launched),
 *     QDWHP_ERR_NOMEM when `ws_bytes` is below the documented size,
 *     QDWHP_ERR_CUDA for a CUDA runtime error (see qdwhp_last_error_message()).
 */
#ifndef QDWHP_H
#define QDWHP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define QDWHP_API __attribute__((visibility("default")))
#else
#define QDWHP_API
#endif

typedef enum {
  QDWHP_OK = 0,
  QDWHP_ERR_ARG = -1,            /* invalid argument */
  QDWHP_ERR_NOMEM = -2,          /* workspace too small */
  QDWHP_ERR_NOT_CONVERGED = -3,  /* Jacobi small solver did not converge in its sweep limit */
  QDWHP_ERR_BREAKDOWN = -4,      /* non-positive pivot in a Cholesky factorisation */
  QDWHP_ERR_NONFINITE = -5,      /* input or an intermediate holds NaN/Inf */
  QDWHP_ERR_TIMEOUT = -6,        /* a bounded wait expired */
  QDWHP_ERR_CUDA = -7,           /* CUDA runtime error */
  QDWHP_ERR_QUEUE_FULL = -8,     /* request queue has no free slot or budget */
  QDWHP_ERR_COUNT = -9,          /* fewer than k wanted pairs captured after the retries */
  QDWHP_PENDING = 1              /* request still running (qdwhp_poll only) */
} qdwhp_status;

typedef enum { QDWHP_LARGEST = 0, QDWHP_SMALLEST = 1 } qdwhp_side;
typedef enum { QDWHP_FP64 = 0, QDWHP_MIXED = 1, QDWHP_FP64_EMULATED = 2, QDWHP_MIXED_EMULATED = 3 } qdwhp_precision;

/* Options.  Fill with qdwhp_default_opts() and change what you need. */
typedef struct {
  int64_t count;          /* wanted count k; 0 = use `fraction` */
  double fraction;        /* k = ceil(fraction * n) (clamped to [1, n]) when count == 0 */
  int32_t side;           /* qdwhp_side (EIG only; SVD always returns the largest) */
  int32_t precision;      /* qdwhp_precision: QDWHP_FP64; QDWHP_MIXED (every Cholesky-based QDWH step
                             but the last in FP32; all else FP64); QDWHP_FP64_EMULATED (every product
                             with m, n >= 128 and k >= 256 by qdwhp_gemm_f64_emulated's scheme, the
                             rest native FP64); QDWHP_MIXED_EMULATED (both) */
  double s_eig;           /* EIG shift / ell_0, Algorithm 1 step 2 (default 0.2) */
  int32_t iters_eig;      /* EIG QDWH iterations (default 3; two for s_eig = 0.875) */
  int32_t lanczos_steps;  /* Lanczos steps for the spectral bounds (default 30, at most 64 used) */
  double tol;             /* index-rule tolerance on |diag(R)|, Section 4.1 (default 0.1; the paper prints 0.01,
                             which holds the FP64 tolerances with use_omega = 1) */
  double c_qr;            /* SVD: QR-based step while c_k > c_qr (default 100) */
  int32_t block_extra;    /* p: the count-to-threshold subspace starts from k + p vectors (16) */
  int32_t power_steps;    /* q: products with the operator; 0 = automatic.  EIG: block Krylov space of
                             depth q (6); SVD: subspace iteration with q + 1 products of A^T A (2) */
  double guard;           /* EIG: minimum wanted width / spectral spread (default 0.10) */
  int32_t max_retries;    /* re-runs with a wider threshold if < k pairs are captured (2) */
  int32_t jacobi_max_sweeps; /* sweep limit of the reduced-problem Jacobi solver (30) */
  uint64_t seed;          /* seed of the SplitMix64 start vectors */
  int32_t refine_steps;   /* SVD: FP64 subspace-iteration steps on Q2, Q2 <- orth(A^T A Q2), before the
                             projection (default 0; for QDWHP_MIXED they restore FP64-level vectors) */
  int32_t zolo_r;         /* 0 (default): QDWH steps.  1..8: Zolo-PD iterations (the type (2r+1, 2r)
                             Zolotarev variant of Section 3.1) from ell_0 = s_eig (EIG) or s (SVD)
                             until ell_k = 1, each with one Gram matrix and r independent terms
                             X (X^T X + c I)^{-1} (Cholesky-formed, or QR-formed when 1 / c > zolo_c_qr);
                             iters_eig is then unused.  QDWHP_FP64 or QDWHP_FP64_EMULATED only. */
  int32_t use_omega;      /* 0 (default) or 1: the extraction QR of Algorithms 1-2 step 3 factors B Omega
                             instead of B (B = (r(A~) + I) / 2, or I - r^T r for the SVD), Omega an n x n
                             Gaussian matrix with N(0, 1/n) entries (SplitMix64 + Box-Muller from `seed`):
                             rank revealing with high probability (Section 4.1), at the cost of one more
                             n x n x n product */
  double zolo_c_qr;       /* Zolo-PD: a term is QR-formed when 1 / c_{2j-1} > zolo_c_qr (default 20) */
} qdwhp_opts;

/* Per-solve report (host struct, filled when the pointer is non-NULL). */
typedef struct {
  int32_t it_qr;          /* QR-based QDWH steps (Zolo-PD: QR-formed terms) */
  int32_t it_chol;        /* Cholesky-based QDWH steps (Zolo-PD: Cholesky-formed terms) */
  int32_t retries;
  int32_t jacobi_sweeps;
  int64_t ell;            /* captured subspace size (n - ind) */
  int64_t k;              /* returned pairs */
  double t;               /* EIG: threshold in the units of A */
  double mu;              /* EIG: lower bound of the shifted matrix (units of A) */
  double s;               /* SVD: relative threshold s */
  double alpha;           /* SVD: estimate of ||A||_2 */
  double ell_k[12];       /* ell_k after each QDWH step */
  double conv[12];        /* ||X_k - X_{k-1}||_F after each QDWH step */
  float ms_total;         /* device time of the solve (CUDA events) */
  int32_t it_f32;         /* Cholesky-based steps run in FP32 (QDWHP_MIXED) */
  int32_t dc_nodes;       /* EIG: spectral splits of the Rayleigh-Ritz problem (0 = Jacobi alone) */
  int32_t zolo_steps;     /* Zolo-PD iterations (0 with QDWH steps) */
} qdwhp_info;

QDWHP_API void qdwhp_default_opts(qdwhp_opts* opts);
QDWHP_API const char* qdwhp_status_string(qdwhp_status s);
/* Text of the last CUDA error seen by this thread ("" if none). */
QDWHP_API const char* qdwhp_last_error_message(void);
/* k = ceil(fraction * n), clamped to [1, n]; 0 if n < 1 or fraction <= 0. */
QDWHP_API int64_t qdwhp_k_from_fraction(int64_t n, double fraction);

/*
 * QDWHpartial-EIG (Algorithm 1; arbitrary side by shift and sign, remark after
 * Algorithm 1): the k largest (side = LARGEST) or smallest eigenpairs of the
 * symmetric n x n matrix A (both triangles must be stored; A is never modified).
 *   lambda: k doubles, ordered largest-first (LARGEST) or smallest-first (SMALLEST).
 *   V:      n x k, leading dimension ldv >= n, orthonormal eigenvectors (signs unspecified).
 *   workspace/ws_bytes: device scratch of at least qdwhp_eig_workspace_bytes(n, opts).
 * k comes from opts->count or opts->fraction.  A spectrum that is one point to rounding
 * (n = 1, c I, the zero matrix) returns the first k unit vectors and their Rayleigh quotients.
 * Errors: QDWHP_ERR_COUNT if fewer than k pairs are captured after opts->max_retries
 * widenings of the threshold; QDWHP_ERR_NONFINITE (A holds NaN/Inf); QDWHP_ERR_BREAKDOWN
 * (a Cholesky-based step failed); QDWHP_ERR_NOT_CONVERGED (the reduced-problem Jacobi hit
 * opts->jacobi_max_sweeps); QDWHP_ERR_ARG for invalid options (nothing launched).
 * Synchronises `stream` (bounds, threshold, ell, counts).
 */
QDWHP_API size_t qdwhp_eig_workspace_bytes(int64_t n, const qdwhp_opts* opts);
QDWHP_API qdwhp_status qdwhp_eig(const double* A, int64_t n, int64_t lda, const qdwhp_opts* opts,
                                 double* lambda, double* V, int64_t ldv,
                                 void* workspace, size_t ws_bytes, qdwhp_info* info, void* stream);

/*
 * QDWHpartial-SVD (Algorithm 2 and the Section 5 listing): the k largest singular
 * triplets of the m x n matrix A (m < n is solved on A^T, Section 4.2).
 *   k: wanted count (0 = take it from opts->count / opts->fraction of min(m, n)).
 *   sigma: k doubles, descending.  U: m x k (ldu >= m).  V: n x k (ldv >= n).
 *   workspace/ws_bytes: at least qdwhp_svd_workspace_bytes(m, n, opts).
 * The zero matrix returns sigma = 0 with the first k unit vectors as U and V.
 * Errors: as for qdwhp_eig; QDWHP_ERR_COUNT also when k exceeds the number of nonzero
 * singular values (only sigma >= s alpha > 0 are kept, Algorithm 2 step 7).
 */
QDWHP_API size_t qdwhp_svd_workspace_bytes(int64_t m, int64_t n, const qdwhp_opts* opts);
QDWHP_API qdwhp_status qdwhp_svd(const double* A, int64_t m, int64_t n, int64_t lda, int64_t k,
                                 const qdwhp_opts* opts, double* sigma, double* U, int64_t ldu,
                                 double* V, int64_t ldv, void* workspace, size_t ws_bytes,
                                 qdwhp_info* info, void* stream);

/*
 * Host-buffer forms of qdwhp_eig and qdwhp_svd (the same solvers): A_host and the outputs are
 * HOST arrays (column-major, leading dimensions as above; page-locked memory lets the copies
 * run asynchronously), the rest as for the device forms.  The library copies A to the device,
 * solves, and copies lambda / sigma, U and V back, all on `stream`, then synchronises it; the
 * outputs are complete on return.  workspace/ws_bytes (device): at least
 * qdwhp_eig_host_workspace_bytes(n, opts) or qdwhp_svd_host_workspace_bytes(m, n, k, opts),
 * which add the device copies of A and of the outputs to the solver's own workspace
 * (0 = invalid sizes).  Errors: as for the device forms; QDWHP_ERR_CUDA if a copy fails.
 */
QDWHP_API size_t qdwhp_eig_host_workspace_bytes(int64_t n, const qdwhp_opts* opts);
QDWHP_API qdwhp_status qdwhp_eig_host(const double* A_host, int64_t n, int64_t lda, const qdwhp_opts* opts,
                                      double* lambda_host, double* V_host, int64_t ldv, void* workspace,
                                      size_t ws_bytes, qdwhp_info* info, void* stream);
QDWHP_API size_t qdwhp_svd_host_workspace_bytes(int64_t m, int64_t n, int64_t k, const qdwhp_opts* opts);
QDWHP_API qdwhp_status qdwhp_svd_host(const double* A_host, int64_t m, int64_t n, int64_t lda, int64_t k,
                                      const qdwhp_opts* opts, double* sigma_host, double* U_host, int64_t ldu,
                                      double* V_host, int64_t ldv, void* workspace, size_t ws_bytes,
                                      qdwhp_info* info, void* stream);

/*
 * Full symmetric eigendecomposition by QDWH spectral divide and conquer (QDWH-EIG,
 * Section 3.2, eq. pdeig): A - sigma I = U_p H, the projector (I + U_p) / 2 splits the
 * spectrum at sigma, and the two Rayleigh-Ritz blocks are split again until they are small
 * enough (order <= 512) for one-sided Jacobi.  sigma is an estimate of the block's median
 * eigenvalue (a midpoint between Gauss-quadrature nodes of 30 Lanczos steps on the block),
 * kept when the split is two-sided and resolved (trace(P) - ||P||_F^2 <= 0.05); otherwise the
 * mean eigenvalue, then the middle of the block's spectral interval.  The same solver handles
 * the Rayleigh-Ritz problems of qdwhp_eig when they are large.
 *   A: n x n symmetric (both triangles stored; the average of A and A^T is used), lda >= n,
 *      never modified.
 *   lambda: n doubles, ascending.  V: n x n (ldv >= n), orthonormal eigenvectors in the
 *      same order (signs unspecified).
 *   workspace/ws_bytes: at least qdwhp_syev_workspace_bytes(n).
 *   Errors: QDWHP_ERR_ARG (bad sizes or pointers, nothing launched), QDWHP_ERR_NOMEM
 *   (workspace too small), QDWHP_ERR_NONFINITE (A holds NaN/Inf), QDWHP_ERR_NOT_CONVERGED
 *   (a Jacobi leaf hit its sweep limit), QDWHP_ERR_BREAKDOWN (a Cholesky-based polar step
 *   failed).  Synchronises `stream` at every split (it reads the split point and rank).
 */
typedef struct {
  int32_t nodes;          /* spectral splits */
  int32_t leaves;         /* Jacobi subproblems */
  int32_t depth;          /* deepest split level */
  int32_t qdwh_steps;     /* polar (QDWH) steps over all splits */
  int32_t refinements;    /* extra subspace-iteration passes beyond the first */
  int32_t jacobi_sweeps;  /* largest sweep count of a leaf */
  double max_offblock;    /* largest ||Q2^T M Q1||_F / ||M - sigma I||_2 of a split */
  float ms_total;         /* device time (CUDA events) */
  int32_t median_splits;  /* splits made at the quadrature median (the others at a fallback point) */
} qdwhp_syev_info;
QDWHP_API size_t qdwhp_syev_workspace_bytes(int64_t n);
QDWHP_API qdwhp_status qdwhp_syev_f64(const double* A, int64_t n, int64_t lda, double* lambda, double* V,
                                      int64_t ldv, void* workspace, size_t ws_bytes, qdwhp_syev_info* info,
                                      void* stream);

/*
 * Full (thin) SVD by QDWH-SVD (Section 3.2): the polar decomposition A = U_p H by QDWH
 * (eqs. practical-polar-qr and practical-polar-chol from ell_0 = 1e-15 on A / alpha, alpha
 * the Lanczos estimate of ||A||_2), the symmetric eigendecomposition H = V Sigma V^T by the
 * divide-and-conquer solver of qdwhp_syev_f64, and U = U_p V.  m < n is solved on A^T with
 * U and V swapped (Section 4.2).  With p = min(m, n):
 *   A: m x n, lda >= m, never modified.
 *   precision: QDWHP_FP64, or QDWHP_FP64_EMULATED (products with m, n >= 128 and k >= 256
 *      emulated on the BF16 tensor cores, as in qdwhp_gemm_f64_emulated); others are
 *      QDWHP_ERR_ARG.
 *   sigma: p doubles, descending.  U: m x p (ldu >= m), V: n x p (ldv >= n), orthonormal
 *      columns (signs unspecified; a sign of U follows its column of V).
 *   The guarantee covers sigma_min / sigma_max >= 1e-15 (the polar factor's ell_0).  If the
 *   smallest computed sigma is at most 1e-14 alpha (numerically rank-deficient A), U is
 *   replaced by the orthonormal factor of its Householder QR, signed by diag(R): the other
 *   columns change only by rounding, the null ones become an orthonormal completion.
 *   workspace/ws_bytes: at least qdwhp_gesvd_workspace_bytes(m, n, precision).
 *   Errors: QDWHP_ERR_ARG, QDWHP_ERR_NOMEM, QDWHP_ERR_NONFINITE (A holds NaN/Inf),
 *   QDWHP_ERR_NOT_CONVERGED, QDWHP_ERR_BREAKDOWN as for qdwhp_syev_f64.  The zero matrix
 *   returns sigma = 0, U and V the leading unit vectors.  Synchronises `stream` (bounds,
 *   the split points of the eigensolver, the smallest sigma).
 */
typedef struct {
  int32_t it_qr;          /* QR-based polar steps (eq. practical-polar-qr) */
  int32_t it_chol;        /* Cholesky-based polar steps (eq. practical-polar-chol) */
  int32_t nodes;          /* spectral splits of the eigensolver on H */
  int32_t leaves;
  int32_t depth;
  int32_t jacobi_sweeps;
  int32_t orthonormalized; /* 1 if U was completed by its QR (numerically rank-deficient A) */
  int32_t median_splits;  /* as in qdwhp_syev_info */
  double alpha;           /* the ||A||_2 estimate A was scaled by */
  double max_offblock;    /* as in qdwhp_syev_info */
  float ms_total;         /* device time (CUDA events) */
} qdwhp_gesvd_info;
QDWHP_API size_t qdwhp_gesvd_workspace_bytes(int64_t m, int64_t n, int32_t precision);
QDWHP_API qdwhp_status qdwhp_gesvd_f64(const double* A, int64_t m, int64_t n, int64_t lda, int32_t precision,
                                       double* sigma, double* U, int64_t ldu, double* V, int64_t ldv,
                                       void* workspace, size_t ws_bytes, qdwhp_gesvd_info* info, void* stream);

/*
 * Launch tuning (not part of the method): per size class (0: <= 128, 1: <= 256, 2: <= 512,
 * 3: <= 1024, 4: larger) the library picks launch shapes from a table that the autotuner
 * (paper_2104_14186_gb300/autotune.py) fills by timing solves.  Every value gives the same
 * result; only the speed changes.  Knobs and their valid ranges:
 *   0  rows per CTA of the cooperative Householder panel, by the panel's row count [16, 512] (64)
 *   1  least warps per CTA of a Jacobi sweep, by the column count                  [1, 16]   (2)
 *   2  CTAs per SM that split-K aims for, by max(m, n) of the product              [1, 8]    (2)
 * qdwhp_tune_set returns QDWHP_ERR_ARG for an unknown knob or class or a value outside the
 * range; qdwhp_tune_get returns -1 for an unknown knob or class.  The table is process-wide;
 * set it before solves start (a solve reads it as it launches).
 */
QDWHP_API qdwhp_status qdwhp_tune_set(int32_t knob, int32_t size_class, int32_t value);
QDWHP_API int32_t qdwhp_tune_get(int32_t knob, int32_t size_class);
QDWHP_API void qdwhp_tune_reset(void);

/* ---- Request queue (serving) and batched solves; not part of the paper's method ---- */

/*
 * A queue runs submitted solves on `max_slots` worker threads, each with its own CUDA
 * stream, inside one device allocation of `hbm_budget_bytes` (the only allocation the
 * library makes; freed by qdwhp_queue_destroy).  A request is admitted when a worker is
 * free and its workspace (qdwhp_eig/svd_workspace_bytes) fits in the unused part of the
 * budget; pending requests are taken oldest first, skipping those that do not fit yet.
 * Requests that arrive while others run start as soon as a slot and memory free up, and
 * their kernels overlap on the device.
 *   `stream` (create): unused, reserved.  `stream` (submit): the caller's stream on which
 *   the input is produced; the solve starts after the work enqueued on it so far.
 *   Inputs and outputs are the caller's device buffers and must stay valid until the
 *   request completes; outputs are complete when qdwhp_poll / qdwhp_wait return OK.
 *   Submit returns QDWHP_ERR_QUEUE_FULL if the request can never fit the budget.
 */
typedef struct qdwhp_queue qdwhp_queue;
QDWHP_API qdwhp_status qdwhp_queue_create(size_t hbm_budget_bytes, int32_t max_slots, void* stream,
                                          qdwhp_queue** q);
QDWHP_API qdwhp_status qdwhp_submit_eig(qdwhp_queue* q, const double* A, int64_t n, int64_t lda,
                                        const qdwhp_opts* opts, double* lambda, double* V, int64_t ldv,
                                        void* stream, uint64_t* req_id);
QDWHP_API qdwhp_status qdwhp_submit_svd(qdwhp_queue* q, const double* A, int64_t m, int64_t n, int64_t lda,
                                        int64_t k, const qdwhp_opts* opts, double* sigma, double* U, int64_t ldu,
                                        double* V, int64_t ldv, void* stream, uint64_t* req_id);
/* QDWHP_PENDING while running; then the request's own status (info filled on completion). */
QDWHP_API qdwhp_status qdwhp_poll(qdwhp_queue* q, uint64_t req_id, qdwhp_info* info);
/* Waits at most timeout_ms (host wait); QDWHP_ERR_TIMEOUT if still running. */
QDWHP_API qdwhp_status qdwhp_wait(qdwhp_queue* q, uint64_t req_id, int32_t timeout_ms, qdwhp_info* info);
/* Host steady-clock seconds of submission, start and completion (QDWHP_PENDING until done). */
QDWHP_API qdwhp_status qdwhp_request_times(qdwhp_queue* q, uint64_t req_id, double* t_submit, double* t_start,
                                           double* t_done);
/* Forgets a completed request (its id becomes invalid). */
QDWHP_API qdwhp_status qdwhp_release(qdwhp_queue* q, uint64_t req_id);
/* Finishes every pending request, joins the workers and frees the budget allocation. */
QDWHP_API qdwhp_status qdwhp_queue_destroy(qdwhp_queue* q);

/*
 * `count` independent QDWHpartial-EIG solves (host arrays of device pointers and sizes;
 * one `opts` for all) run `concurrency` at a time through a queue sized for the largest
 * workspaces, largest problems first.  statuses[i] (and infos[i], if non-NULL) per
 * problem; returns the first error, if any.  Allocates (and frees) the queue's budget.
 */
QDWHP_API qdwhp_status qdwhp_eig_batched(int64_t count, const double* const* A, const int64_t* n,
                                         const int64_t* lda, const qdwhp_opts* opts, double* const* lambda,
                                         double* const* V, const int64_t* ldv, int32_t concurrency,
                                         qdwhp_status* statuses, qdwhp_info* infos, void* stream);

/* ---- Building blocks (the dense kernels the solvers are made of) ---- */

/*
 * C = alpha * op(A) * op(B) + beta * C, FP64 (op = transpose when trans != 0);
 * C is m x n, the inner dimension k.  beta == 0 never reads C.  The products in
 * the Cholesky-based QDWH step (eq. practical-polar-chol), the Householder
 * trailing updates and the Rayleigh-Ritz projections (Algorithms 1-2) are these.
 */
QDWHP_API qdwhp_status qdwhp_gemm_f64(int transa, int transb, int64_t m, int64_t n, int64_t k,
                                      double alpha, const double* A, int64_t lda,
                                      const double* B, int64_t ldb, double beta,
                                      double* C, int64_t ldc, void* stream);

/*
 * The same product, FP64-accurate, computed on the BF16 tensor cores by the Ozaki splitting
 * scheme (Ozaki, Ogita, Oishi, Rump 2012): each row of op(A) and column of op(B) is scaled
 * by a power of two and cut into nine 6-bit digits; the 60 digit products with
 * s + t <= 12 are exact in FP32 and summed in FP64.  The error is normwise, relative to the
 * largest entry of each row of op(A) and column of op(B): about 2^-54 of those, plus FP64
 * rounding of the sum.  Not part of the paper.
 *   workspace/ws_bytes: at least qdwhp_gemm_f64_emulated_workspace_bytes(m, n, k), 16-byte
 *   aligned.  A NaN or Inf in a row of op(A) or a column of op(B) makes that row or column
 *   of the result NaN.
 */
QDWHP_API size_t qdwhp_gemm_f64_emulated_workspace_bytes(int64_t m, int64_t n, int64_t k);
QDWHP_API qdwhp_status qdwhp_gemm_f64_emulated(int transa, int transb, int64_t m, int64_t n, int64_t k,
                                               double alpha, const double* A, int64_t lda,
                                               const double* B, int64_t ldb, double beta,
                                               double* C, int64_t ldc, void* workspace, size_t ws_bytes,
                                               void* stream);

/*
 * C = alpha * op(A) * op(B) + beta * C in FP32 (A, B, C float, column-major), FP32-accurate, on
 * the BF16 tensor cores: each entry is split into three bfloat16 slices (x = h + m + l, each the
 * rounding of what the previous ones leave), the six slice products with s + t <= 2 run as
 * tcgen05 MMAs into one FP32 accumulator, so the error is that of an FP32 product (about 2^-24
 * relative per term plus FP32 rounding of the sums).  Not part of the paper: the products of the
 * FP32 Cholesky-based QDWH steps (eq. practical-polar-chol) of QDWHP_MIXED run on it.
 *   workspace/ws_bytes: at least qdwhp_gemm_f32_bf16x6_workspace_bytes(m, n, k), 16-byte aligned.
 *   beta == 0 never reads C.  A NaN or Inf in op(A) or op(B) reaches the affected rows and columns.
 */
QDWHP_API size_t qdwhp_gemm_f32_bf16x6_workspace_bytes(int64_t m, int64_t n, int64_t k);
QDWHP_API qdwhp_status qdwhp_gemm_f32_bf16x6(int transa, int transb, int64_t m, int64_t n, int64_t k, float alpha,
                                             const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                                             float* C, int64_t ldc, void* workspace, size_t ws_bytes, void* stream);

/*
 * Z = L L^T, lower Cholesky factor of the symmetric positive definite n x n Z in
 * place (lower triangle read and written; the strict upper triangle is left as is).
 * The factorisation W = chol(Z) of eq. practical-polar-chol with W = L^T.
 * *info_host = 0 on success, i > 0 if the leading minor of order i is not
 * positive definite (status QDWHP_ERR_BREAKDOWN).  Synchronises `stream`.
 */
QDWHP_API size_t qdwhp_potrf_workspace_bytes(int64_t n);
QDWHP_API qdwhp_status qdwhp_potrf_f64(int64_t n, double* Z, int64_t ldz, void* workspace, size_t ws_bytes,
                                       int* info_host, void* stream);

/*
 * Householder QR (unpivoted, as in Algorithm 1 step 3) of the m x n matrix A,
 * m >= n: A = Q R with Q m x n orthonormal and R n x n upper triangular, written
 * to Q (ldq >= m) and R (ldr >= n).  A is overwritten.  diag(R) follows the
 * Householder convention R_ii = -sign(a_ii) * ||a_i||.
 */
QDWHP_API size_t qdwhp_qr_workspace_bytes(int64_t m, int64_t n);
QDWHP_API qdwhp_status qdwhp_qr_f64(int64_t m, int64_t n, double* A, int64_t lda, double* Q, int64_t ldq,
                                    double* R, int64_t ldr, void* workspace, size_t ws_bytes, void* stream);

/*
 * QDWH steps in place on the m x n iterate X (m >= n): for step i with weights
 * (a, b, c) = abc_host[3i .. 3i+2], the QR-based update of eq. practical-polar-qr
 * if use_qr_host[i] != 0, else the Cholesky-based update of eq. practical-polar-chol.
 * conv_host (may be NULL) receives ||X_i - X_{i-1}||_F per step.
 */
QDWHP_API size_t qdwhp_qdwh_workspace_bytes(int64_t m, int64_t n);
QDWHP_API qdwhp_status qdwhp_qdwh_steps_f64(int64_t m, int64_t n, double* X, int64_t ldx, int32_t nsteps,
                                            const double* abc_host, const int32_t* use_qr_host,
                                            double* conv_host, void* workspace, size_t ws_bytes,
                                            void* stream);

/*
 * Cholesky factorisation with no workspace argument; it allocates no memory.
 * The paper has no counterpart: this is a convenience for callers that cannot give
 * the library device scratch, e.g. a program whose device memory belongs to another
 * allocator (a framework's caching pool, a server's fixed memory plan) and must not
 * call cudaMalloc behind its back, or code that cannot afford the device-wide
 * synchronisation a cudaMalloc/cudaFree may cause.
 *   Same result as qdwhp_potrf_f64 (same arguments minus the workspace).
 *   n <= QDWHP_POTRF_NOALLOC_MAX_N, else QDWHP_ERR_ARG with a message in
 *   qdwhp_last_error_message() and nothing launched.
 *   Scratch: a 4 MB array in the library's own device memory, held by every GPU that
 *   loads the library until the process exits.  The first call on a device looks up
 *   that array's device address (with the device current).  All calls share the one
 *   array, so calls that overlap on the GPU (other streams, other host threads) race:
 *   serialise them.
 *   Every call synchronises `stream` to read the result flag, so the entry point cannot
 *   be used inside a stream capture at all.
 */
#define QDWHP_POTRF_NOALLOC_MAX_N 4096
QDWHP_API qdwhp_status qdwhp_potrf_f64_noalloc(int64_t n, double* Z, int64_t ldz, int* info_host, void* stream);

/* ---- Instrumentation (not part of the method) ---- */

/* Kernels launched by this library since it was loaded (all threads). */
QDWHP_API unsigned long long qdwhp_launch_count(void);
/*
 * Opt-in timing of the FP64 GEMM launches: between qdwhp_profile_begin() and
 * qdwhp_profile_end(), every GEMM the library launches is bracketed by CUDA events on
 * its stream; qdwhp_profile_end() waits for them and returns the summed device time
 * (ms), the summed algorithmic flops (2mnk, or n(n+1)k for a lower-triangular
 * product) and the number of GEMMs.  Process-wide; use from one host thread.
 */
QDWHP_API qdwhp_status qdwhp_profile_begin(void);
QDWHP_API qdwhp_status qdwhp_profile_end(double* gemm_ms, double* gemm_flops, int64_t* gemm_launches);
/* Per-GEMM records of the last profile: 6 doubles each (m, n, k, lower-triangle flag,
 * split-K slices, ms), up to `capacity` records into `out` (host); returns the count. */
QDWHP_API int64_t qdwhp_profile_records(double* out, int64_t capacity);

#ifdef __cplusplus
}
#endif

#endif /* QDWHP_H */
