// Cholesky factorisation and right-side triangular solves for the Cholesky-based
// QDWH step (eq. practical-polar-chol): W = chol(Z) is kept as L = W^T in the lower
// triangle, and X W^{-1} W^{-T} = (X L^{-T}) L^{-1}.
//
// Both are recursive (split the order in two halves at a multiple of kCholNB), so
// almost all flops land in large DMMA GEMMs.  The kCholNB x kCholNB diagonal leaves
// are factored by one CTA in shared memory, which also writes the inverse of each
// leaf; the triangular solves then apply those inverses as small GEMMs instead of
// running a sequential substitution.
#include <mutex>

#include "internal.h"

namespace qdwhp {

namespace {

constexpr int NB = kCholNB;

// One diagonal leaf: Z (nb x nb, lower) -> L with Z = L L^T, plus inv(L) (lower) into Linv (ld NB).
// Right-looking in shared memory; each pivot's reciprocal is formed once so the column
// scaling and the inverse use multiplies.  inv(L) is formed by the same right-looking
// substitution applied to all columns of the identity at once (parallel over entries).
template <typename T>
constexpr size_t leaf_smem() { return 2 * sizeof(T) * NB * (NB + 1) + sizeof(T) * NB; }

template <typename T>
__global__ void __launch_bounds__(256) potrf_leaf_kernel(int nb, T* Z, int64_t ldz, T* Linv, int* fail,
                                                         int col_offset) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  T (*a)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(sm);
  T (*x)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(sm + NB * (NB + 1));
  T* dinv = sm + 2 * NB * (NB + 1);
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int i = e % NB, j = e / NB;
    a[i][j] = (i < nb && j < nb && i >= j) ? Z[i + (int64_t)j * ldz] : T(0);
    x[i][j] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      T d = a[j][j];
      if (!(d > T(0)) || !isfinite(d)) {
        atomicCAS(fail, 0, col_offset + j + 1);
        d = T(1);
      }
      const T piv = sqrt(d);
      a[j][j] = piv;
      dinv[j] = T(1) / piv;
    }
    __syncthreads();
    const T r = dinv[j];
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) a[i][j] *= r;
    __syncthreads();
    const int rem = nb - j - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e % rem, c = j + 1 + e / rem;
      if (i >= c) a[i][c] -= a[i][j] * a[c][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e % nb, j = e / nb;
    if (i >= j) Z[i + (int64_t)j * ldz] = a[i][j];
  }
  // Solve L X = I: for each j, row j of X is scaled by 1/L_jj, then eliminated from rows below.
  for (int j = 0; j < nb; ++j) {
    const T r = dinv[j];
    for (int c = tid; c <= j; c += blockDim.x) x[j][c] *= r;
    __syncthreads();
    const int rem = nb - j - 1;
    for (int e = tid; e < rem * (j + 1); e += blockDim.x) {
      const int i = j + 1 + e % rem, c = e / rem;
      x[i][c] -= a[i][j] * x[j][c];
    }
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int i = e % NB, j = e / NB;
    Linv[i + (int64_t)j * NB] = (i < nb && j < nb) ? x[i][j] : T(0);
  }
}

inline int64_t split_point(int64_t n) {
  int64_t n1 = ((n / 2) / NB) * NB;
  return n1 == 0 ? NB : n1;
}

template <typename T>
qdwhp_status trsm_rec(cudaStream_t st, bool trans, int64_t m, int64_t n, T* X, int64_t ldx, const T* L, int64_t ldl,
                      const T* Linv, T* scratch) {
  if (n <= NB) {
    // X := X inv(L_b)^T (trans) or X inv(L_b), through a scratch copy.
    QDWHP_TRY(gemm(st, false, trans, m, n, n, T(1), X, ldx, Linv, NB, T(0), scratch, m));
    return copy_matrix(st, m, n, scratch, m, X, ldx);
  }
  const int64_t n1 = split_point(n), n2 = n - n1;
  T* X1 = X;
  T* X2 = X + n1 * ldx;
  const T* L21 = L + n1;
  const T* L22 = L + n1 + n1 * ldl;
  const T* Linv2 = Linv + (n1 / NB) * NB * NB;
  if (trans) {
    // [Y1 Y2] [L11^T L21^T; 0 L22^T] = [X1 X2]
    QDWHP_TRY(trsm_rec<T>(st, true, m, n1, X1, ldx, L, ldl, Linv, scratch));
    QDWHP_TRY(gemm(st, false, true, m, n2, n1, T(-1), X1, ldx, L21, ldl, T(1), X2, ldx));
    return trsm_rec<T>(st, true, m, n2, X2, ldx, L22, ldl, Linv2, scratch);
  }
  // [Y1 Y2] [L11 0; L21 L22] = [X1 X2]
  QDWHP_TRY(trsm_rec<T>(st, false, m, n2, X2, ldx, L22, ldl, Linv2, scratch));
  QDWHP_TRY(gemm(st, false, false, m, n1, n2, T(-1), X2, ldx, L21, ldl, T(1), X1, ldx));
  return trsm_rec<T>(st, false, m, n1, X1, ldx, L, ldl, Linv, scratch);
}

template <typename T>
qdwhp_status potrf_rec(cudaStream_t st, int64_t n, T* Z, int64_t ldz, T* Linv, T* scratch, int* fail, int64_t off) {
  if (n <= NB) {
    static PerDeviceOnce attr;
    QDWHP_CUDA_TRY(attr.run([] {
      return cudaFuncSetAttribute(potrf_leaf_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)leaf_smem<T>());
    }));
    potrf_leaf_kernel<T><<<1, 256, leaf_smem<T>(), st>>>((int)n, Z, ldz, Linv, fail, (int)off);
    QDWHP_LAUNCH_CHECK();
    return QDWHP_OK;
  }
  const int64_t n1 = split_point(n), n2 = n - n1;
  T* Z21 = Z + n1;
  T* Z22 = Z + n1 + n1 * ldz;
  QDWHP_TRY(potrf_rec<T>(st, n1, Z, ldz, Linv, scratch, fail, off));
  // L21 = Z21 L11^{-T}
  QDWHP_TRY(trsm_rec<T>(st, true, n2, n1, Z21, ldz, Z, ldz, Linv, scratch));
  // Z22 -= L21 L21^T (lower triangle)
  QDWHP_TRY(gemm(st, false, true, n2, n2, n1, T(-1), Z21, ldz, Z21, ldz, T(1), Z22, ldz, LOWER));
  return potrf_rec<T>(st, n2, Z22, ldz, Linv + (n1 / NB) * NB * NB, scratch, fail, off + n1);
}

}  // namespace

size_t potrf_linv_elems(int64_t n) { return (size_t)((n + NB - 1) / NB) * NB * NB; }
size_t potrf_scratch_elems(int64_t n) { return (size_t)std::max<int64_t>(n, 1) * NB; }
size_t trsm_scratch_elems(int64_t m, int64_t n) { (void)n; return (size_t)std::max<int64_t>(m, 1) * NB; }

qdwhp_status potrf(cudaStream_t st, int64_t n, double* Z, int64_t ldz, double* Linv, double* scratch,
                   int* fail_dev) {
  if (n <= 0) return QDWHP_OK;
  return potrf_rec<double>(st, n, Z, ldz, Linv, scratch, fail_dev, 0);
}

qdwhp_status potrf(cudaStream_t st, int64_t n, float* Z, int64_t ldz, float* Linv, float* scratch, int* fail_dev) {
  if (n <= 0) return QDWHP_OK;
  return potrf_rec<float>(st, n, Z, ldz, Linv, scratch, fail_dev, 0);
}

qdwhp_status trsm_right_lower(cudaStream_t st, bool trans, int64_t m, int64_t n, double* X, int64_t ldx,
                              const double* L, int64_t ldl, const double* Linv, double* scratch) {
  if (m <= 0 || n <= 0) return QDWHP_OK;
  return trsm_rec<double>(st, trans, m, n, X, ldx, L, ldl, Linv, scratch);
}

qdwhp_status trsm_right_lower(cudaStream_t st, bool trans, int64_t m, int64_t n, float* X, int64_t ldx,
                              const float* L, int64_t ldl, const float* Linv, float* scratch) {
  if (m <= 0 || n <= 0) return QDWHP_OK;
  return trsm_rec<float>(st, trans, m, n, X, ldx, L, ldl, Linv, scratch);
}

}  // namespace qdwhp
