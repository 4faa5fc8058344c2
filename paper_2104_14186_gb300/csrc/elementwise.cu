// Memory-bound helpers: axpby (the QDWH update's combination step), copies,
// identity shifts, symmetrisation and reductions.  All are grid-stride loops over
// column-major matrices with grids sized in multiples of the SM count.
#include "internal.h"

namespace qdwhp {

namespace {

inline int grid_for(size_t total) {
  return (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, 8 * (size_t)kNumSMs));
}

template <typename T>
__global__ void axpby_kernel(int M, int N, T alpha, const T* X, int64_t ldx, T beta, T* Y, int64_t ldy, T diag_add) {
  const size_t total = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % M), j = (int)(e / M);
    T v = alpha * X[i + (int64_t)j * ldx];
    T* yp = Y + i + (int64_t)j * ldy;
    if (beta != T(0)) v += beta * (*yp);
    if (i == j) v += diag_add;
    *yp = v;
  }
}

template <typename T>
__global__ void axpby_diff_kernel(int M, int N, T a, T* Y, int64_t ldy, T b, const T* Z, int64_t ldz,
                                  double* diff_part) {
  __shared__ double red[32];
  const size_t total = (size_t)M * N;
  double acc = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % M), j = (int)(e / M);
    T* yp = Y + i + (int64_t)j * ldy;
    const T old = *yp;
    const T nw = a * old + b * Z[i + (int64_t)j * ldz];
    *yp = nw;
    const double d = (double)nw - (double)old;
    acc += d * d;
  }
  acc = block_sum(acc, red);
  if (diff_part != nullptr && threadIdx.x == 0) diff_part[blockIdx.x] = acc;
}

template <typename T>
__global__ void set_kernel(int M, int N, T off, T diag, T* Y, int64_t ldy) {
  const size_t total = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % M), j = (int)(e / M);
    Y[i + (int64_t)j * ldy] = (i == j) ? diag : off;
  }
}

template <typename S, typename D>
__global__ void convert_kernel(int M, int N, const S* X, int64_t ldx, D* Y, int64_t ldy) {
  const size_t total = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % M), j = (int)(e / M);
    Y[i + (int64_t)j * ldy] = (D)X[i + (int64_t)j * ldx];
  }
}

__global__ void copy_upper_kernel(int N, const double* A, int64_t lda, double* R, int64_t ldr) {
  const size_t total = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % N), j = (int)(e / N);
    R[i + (int64_t)j * ldr] = (i <= j) ? A[i + (int64_t)j * lda] : 0.0;
  }
}

// B (cols x rows) = A^T (rows x cols), through 32 x 33 shared tiles.
__global__ void transpose_kernel(int rows, int cols, const double* A, int64_t lda, double* B, int64_t ldb) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int i = bx + threadIdx.x, j = by + k;
    if (i < rows && j < cols) tile[k][threadIdx.x] = A[i + (int64_t)j * lda];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int i = by + threadIdx.x, j = bx + k;   // B(i, j) = A(j, i)
    if (i < cols && j < rows) B[i + (int64_t)j * ldb] = tile[threadIdx.x][k];
  }
}

// G = R^T for the upper triangle R of A (the strictly lower part of G is R's upper part).
__global__ void copy_upper_t_kernel(int N, const double* A, int64_t lda, double* G, int64_t ldg) {
  const size_t total = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % N), j = (int)(e / N);
    G[i + (int64_t)j * ldg] = (j <= i) ? A[j + (int64_t)i * lda] : 0.0;
  }
}

__global__ void symmetrize_avg_kernel(int n, double* H, int64_t ldh) {
  const size_t total = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i < j) {
      const double v = 0.5 * (H[i + (int64_t)j * ldh] + H[j + (int64_t)i * ldh]);
      H[i + (int64_t)j * ldh] = v;
      H[j + (int64_t)i * ldh] = v;
    }
  }
}

__global__ void symmetrize_kernel(int N, double* Y, int64_t ldy) {
  const size_t total = (size_t)N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % N), j = (int)(e / N);
    if (i < j) Y[i + (int64_t)j * ldy] = Y[j + (int64_t)i * ldy];
  }
}

__global__ void reduce_parts_kernel(const double* parts, int nparts, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += parts[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) *out = acc;
}

__global__ void nonfinite_kernel(int M, int N, const double* X, int64_t ldx, unsigned* count) {
  const size_t total = (size_t)M * N;
  unsigned c = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % M), j = (int)(e / M);
    if (!isfinite(X[i + (int64_t)j * ldx])) ++c;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

}  // namespace

template <typename T>
qdwhp_status axpby_t(cudaStream_t st, int64_t m, int64_t n, T alpha, const T* X, int64_t ldx, T beta, T* Y,
                     int64_t ldy, T diag_add) {
  if (m <= 0 || n <= 0) return QDWHP_OK;
  axpby_kernel<T><<<grid_for((size_t)m * n), 256, 0, st>>>((int)m, (int)n, alpha, X, ldx, beta, Y, ldy, diag_add);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status axpby(cudaStream_t st, int64_t m, int64_t n, double alpha, const double* X, int64_t ldx, double beta,
                   double* Y, int64_t ldy, double diag_add) {
  return axpby_t<double>(st, m, n, alpha, X, ldx, beta, Y, ldy, diag_add);
}
qdwhp_status axpby(cudaStream_t st, int64_t m, int64_t n, float alpha, const float* X, int64_t ldx, float beta,
                   float* Y, int64_t ldy, float diag_add) {
  return axpby_t<float>(st, m, n, alpha, X, ldx, beta, Y, ldy, diag_add);
}

template <typename T>
qdwhp_status axpby_diff_t(cudaStream_t st, int64_t m, int64_t n, T a, T* Y, int64_t ldy, T b, const T* Z,
                          int64_t ldz, double* diff_part) {
  if (m <= 0 || n <= 0) return QDWHP_OK;
  // Exactly kDiffParts blocks so that every partial slot is written.
  axpby_diff_kernel<T><<<kDiffParts, 256, 0, st>>>((int)m, (int)n, a, Y, ldy, b, Z, ldz, diff_part);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status axpby_diff(cudaStream_t st, int64_t m, int64_t n, double a, double* Y, int64_t ldy, double b,
                        const double* Z, int64_t ldz, double* diff_part) {
  return axpby_diff_t<double>(st, m, n, a, Y, ldy, b, Z, ldz, diff_part);
}
qdwhp_status axpby_diff(cudaStream_t st, int64_t m, int64_t n, float a, float* Y, int64_t ldy, float b,
                        const float* Z, int64_t ldz, double* diff_part) {
  return axpby_diff_t<float>(st, m, n, a, Y, ldy, b, Z, ldz, diff_part);
}

template <typename T>
qdwhp_status copy_matrix_t(cudaStream_t st, int64_t m, int64_t n, const T* X, int64_t ldx, T* Y, int64_t ldy) {
  if (m <= 0 || n <= 0) return QDWHP_OK;
  if (ldx == m && ldy == m) {
    QDWHP_CUDA_TRY(cudaMemcpyAsync(Y, X, sizeof(T) * m * n, cudaMemcpyDeviceToDevice, st));
    return QDWHP_OK;
  }
  QDWHP_CUDA_TRY(cudaMemcpy2DAsync(Y, sizeof(T) * ldy, X, sizeof(T) * ldx, sizeof(T) * m, n,
                                   cudaMemcpyDeviceToDevice, st));
  return QDWHP_OK;
}

qdwhp_status copy_matrix(cudaStream_t st, int64_t m, int64_t n, const double* X, int64_t ldx, double* Y,
                         int64_t ldy) {
  return copy_matrix_t<double>(st, m, n, X, ldx, Y, ldy);
}
qdwhp_status copy_matrix(cudaStream_t st, int64_t m, int64_t n, const float* X, int64_t ldx, float* Y, int64_t ldy) {
  return copy_matrix_t<float>(st, m, n, X, ldx, Y, ldy);
}

template <typename T>
qdwhp_status set_matrix_t(cudaStream_t st, int64_t m, int64_t n, T off, T diag, T* Y, int64_t ldy) {
  if (m <= 0 || n <= 0) return QDWHP_OK;
  set_kernel<T><<<grid_for((size_t)m * n), 256, 0, st>>>((int)m, (int)n, off, diag, Y, ldy);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status set_matrix(cudaStream_t st, int64_t m, int64_t n, double off, double diag, double* Y, int64_t ldy) {
  return set_matrix_t<double>(st, m, n, off, diag, Y, ldy);
}
qdwhp_status set_matrix(cudaStream_t st, int64_t m, int64_t n, float off, float diag, float* Y, int64_t ldy) {
  return set_matrix_t<float>(st, m, n, off, diag, Y, ldy);
}

qdwhp_status convert(cudaStream_t st, int64_t m, int64_t n, const double* X, int64_t ldx, float* Y, int64_t ldy) {
  if (m <= 0 || n <= 0) return QDWHP_OK;
  convert_kernel<double, float><<<grid_for((size_t)m * n), 256, 0, st>>>((int)m, (int)n, X, ldx, Y, ldy);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}
qdwhp_status convert(cudaStream_t st, int64_t m, int64_t n, const float* X, int64_t ldx, double* Y, int64_t ldy) {
  if (m <= 0 || n <= 0) return QDWHP_OK;
  convert_kernel<float, double><<<grid_for((size_t)m * n), 256, 0, st>>>((int)m, (int)n, X, ldx, Y, ldy);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status copy_upper(cudaStream_t st, int64_t n, const double* A, int64_t lda, double* R, int64_t ldr) {
  if (n <= 0) return QDWHP_OK;
  copy_upper_kernel<<<grid_for((size_t)n * n), 256, 0, st>>>((int)n, A, lda, R, ldr);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status transpose(cudaStream_t st, int64_t rows, int64_t cols, const double* A, int64_t lda, double* B,
                       int64_t ldb) {
  if (rows <= 0 || cols <= 0) return QDWHP_OK;
  dim3 grid(ceil_div(rows, 32), ceil_div(cols, 32));
  transpose_kernel<<<grid, dim3(32, 8), 0, st>>>((int)rows, (int)cols, A, lda, B, ldb);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status symmetrize_avg(cudaStream_t st, int64_t n, double* H, int64_t ldh) {
  if (n <= 1) return QDWHP_OK;
  const size_t total = (size_t)n * n;
  symmetrize_avg_kernel<<<(int)std::min<size_t>((total + 255) / 256, 8 * kNumSMs), 256, 0, st>>>((int)n, H, ldh);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status copy_upper_t(cudaStream_t st, int64_t n, const double* A, int64_t lda, double* G, int64_t ldg) {
  if (n <= 0) return QDWHP_OK;
  copy_upper_t_kernel<<<grid_for((size_t)n * n), 256, 0, st>>>((int)n, A, lda, G, ldg);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status symmetrize_from_lower(cudaStream_t st, int64_t n, double* Y, int64_t ldy) {
  if (n <= 1) return QDWHP_OK;
  symmetrize_kernel<<<grid_for((size_t)n * n), 256, 0, st>>>((int)n, Y, ldy);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status reduce_parts(cudaStream_t st, const double* parts, int nparts, double* out) {
  reduce_parts_kernel<<<1, 1024, 0, st>>>(parts, nparts, out);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

qdwhp_status count_nonfinite(cudaStream_t st, int64_t m, int64_t n, const double* X, int64_t ldx,
                             unsigned* count_dev) {
  if (m <= 0 || n <= 0) return QDWHP_OK;
  nonfinite_kernel<<<grid_for((size_t)m * n), 256, 0, st>>>((int)m, (int)n, X, ldx, count_dev);
  QDWHP_LAUNCH_CHECK();
  return QDWHP_OK;
}

}  // namespace qdwhp
