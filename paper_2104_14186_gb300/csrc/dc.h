// Internal interface of dc.cu: symmetric eigendecomposition by QDWH spectral divide and
// conquer (QDWH-EIG, Section 3.2), the reduced eigensolver for large Rayleigh-Ritz problems
// and the full-spectrum entry point.
#pragma once

#include "internal.h"
#include "krylov.h"
#include "qdwh.h"

namespace qdwhp {

// Subproblems up to this order go to one-sided Jacobi (leaves); larger ones are split.
constexpr int64_t kDcLeaf = 512;
// Rayleigh-Ritz problems of the partial solvers switch from Jacobi to divide and conquer
// above this order (the workspace of a solve of order n > kDcMin holds the extra buffers).
constexpr int64_t kDcMin = 1024;
// ell_0 of every split's polar decomposition: eigenvalues closer to the split point than
// kDcEll0 * ||M - sigma I||_2 are not separated, and either side is then backward stable.
constexpr double kDcEll0 = 1e-15;

struct DcWs {
  int64_t cap = 0;
  double* M = nullptr;   // cap^2: node matrices; a node's children overwrite its slot
  double* X = nullptr;   // cap^2: polar iterate, then the spectral projector P
  double* Q = nullptr;   // cap^2: random start block, then the split basis [Q1 Q2]; leaf Jacobi vectors
  double* W = nullptr;   // cap^2: P Omega, M Q, V Q; leaf G
  double* E = nullptr;   // cap^2 / 4 (+ slack): off-diagonal block Q2^T M Q1
  QRFactors f;           // reflectors of the n x r block (cap x cap capacity)
  double* qr_scratch = nullptr;
  QdwhWs q;              // polar decomposition with QR-based steps (cap x cap)
  Schedule* sched = nullptr;
  double* scal = nullptr;    // device scalars
  double* parts = nullptr;   // kDiffParts partial sums
  JacobiState* jst = nullptr;
  LanczosState* lst = nullptr;   // split-point estimate: Lanczos on the node matrix
  double* lws = nullptr;
};

// Carves every buffer of w for problems up to order cap.
void carve_dc(Arena& ar, int64_t cap, DcWs& w);
// Carves only E, q and the small buffers; the caller points M, X, Q, W (cap^2 each), f (a
// cap x cap QR) and qr_scratch (qr_scratch_elems(cap, cap)) at memory it lends.
void carve_dc_own(Arena& ar, int64_t cap, DcWs& w);

struct DcStats {
  int nodes = 0;           // split nodes
  int leaves = 0;
  int depth = 0;           // deepest split level
  int qdwh_steps = 0;      // polar steps over all nodes
  int refinements = 0;     // extra subspace-iteration passes (off-diagonal block above tolerance)
  int jacobi_sweeps = 0;   // largest leaf sweep count
  double max_offblock = 0; // largest ||Q2^T M Q1||_F / ||M - sigma I||_2 accepted
  int median_splits = 0;   // splits made at the quadrature estimate of the median
  int unresolved_splits = 0; // candidate split points rejected: eigenvalues within the polar resolution
};

// Eigendecomposition of the symmetric n x n matrix held in w.M (ld n; destroyed), whose
// spectrum lies in [lo, hi].  lam (device, n) receives the eigenvalues (unordered); with
// `vectors`, V (n x n, ld ldv) the orthonormal eigenvectors in the same order.  Without
// `vectors` only the eigenvalues are computed (no back-transformations, looser leaf Jacobi).
qdwhp_status sym_eig_dc(cudaStream_t st, int64_t n, double lo, double hi, uint64_t seed, bool vectors,
                        int jacobi_max_sweeps, double* lam, double* V, int64_t ldv, DcWs& w, DcStats* stats);

// ---- gesvd.cu ----
// All singular triplets of the n x n R by QDWH-SVD (polar factor, divide-and-conquer eigensolver
// of H = U_p^T R, U = U_p V), for the reduced problem of the partial SVD: sigma (n) descending,
// U (n x n, ld ldu; may be the storage of R, which is read only before U is written) and V
// (n x n, ld ldv).  `ws` holds gesvd_square_ws_bytes(n) bytes; *sweeps gets the largest Jacobi
// sweep count of the eigensolver's leaves.
size_t gesvd_square_ws_bytes(int64_t n);
qdwhp_status gesvd_square(cudaStream_t st, int64_t n, const double* R, int64_t ldr, double* sigma, double* U,
                          int64_t ldu, double* V, int64_t ldv, void* ws, size_t ws_bytes, int* sweeps);

}  // namespace qdwhp
