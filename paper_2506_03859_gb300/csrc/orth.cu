// Orthonormalisation and reduction kernels of the farPCA block (arxiv
// 2506.03859): the b x b Cholesky factor of a Gram matrix and its inverse (the
// basis Q_j = Y' R^{-1}, the role of Z^{-1} in Alg. 1 step 10), the Frobenius
// norms behind the error indicator (E = ||A||_F^2 - sum_j ||B_j||_F^2, Sec. 2.1),
// and the row append of B_j.  All reductions use a fixed order so repeated runs
// give identical bits.
#include <math.h>

#include "chol.cuh"
#include "internal.cuh"

namespace lra {

__device__ __forceinline__ double block_sum_256(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
  __syncthreads();
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(256) k_col_sums(const double* __restrict__ X, int64_t ld,
                                                  int64_t rows, double* __restrict__ sumsq,
                                                  double* __restrict__ sum) {
  __shared__ double red[8];
  const int64_t c = blockIdx.x;
  const double* col = X + c * ld;
  double sq = 0.0, s = 0.0;
  for (int64_t i = threadIdx.x; i < rows; i += 256) {
    const double x = __ldg(col + i);
    sq = fma(x, x, sq);
    s += x;
  }
  if (sumsq) {
    const double t = block_sum_256(sq, red);
    if (threadIdx.x == 0) sumsq[c] = t;
  }
  if (sum) {
    const double t = block_sum_256(s, red);
    if (threadIdx.x == 0) sum[c] = t;
  }
}

// One pass over A (m x n, column-major) for the set-up of a run: per-column sums of
// squares (||A||_F^2 of Alg. 1 step 1, summed per column over 512-row blocks,
// then over the blocks in order), and the largest biased exponent of every
// column and every row (the scales of the tensor-core digits).  CTA (rb, cb):
// rows 512 rb .., columns 32 cb ..; warp w takes 4 of the columns, lane l the
// rows l, l + 32, ...; per column the warp reduces by shuffles; row maxima meet
// in shared memory, one atomic per row and CTA.  colE and rowE start at zero.
// T: element type of A (float entries are converted exactly to double on load).
template <typename T>
__global__ void __launch_bounds__(256) k_a_stats(const T* __restrict__ A, int64_t lda,
                                                 int64_t m, int64_t n, double* __restrict__ part,
                                                 int* __restrict__ colE, int* __restrict__ rowE) {
  __shared__ int srow[8][512];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * 512, c0 = (int64_t)blockIdx.y * 32 + warp * 4;
  int rmax[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) rmax[k] = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t c = c0 + q;
    if (c >= n) break;  // warp-uniform
    const T* col = A + c * lda + r0;
    double s0 = 0.0, s1 = 0.0;
    int e = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int64_t r = lane + 32 * k;
      const double x = (r0 + r < m) ? (double)__ldg(col + r) : 0.0;
      const int ex = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
      e = max(e, ex);
      rmax[k] = max(rmax[k], ex);
      if (k & 1)
        s1 = fma(x, x, s1);
      else
        s0 = fma(x, x, s0);
    }
    double sq = s0 + s1;
    for (int o = 16; o > 0; o >>= 1) {
      sq += __shfl_down_sync(0xffffffffu, sq, o);
      e = max(e, __shfl_down_sync(0xffffffffu, e, o));
    }
    if (lane == 0) {
      part[(int64_t)blockIdx.x * n + c] = sq;
      atomicMax(colE + c, e);
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) srow[warp][lane + 32 * k] = rmax[k];
  __syncthreads();
  for (int r = threadIdx.x; r < 512; r += 256) {
    int e = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) e = max(e, srow[w][r]);
    if (r0 + r < m) atomicMax(rowE + r0 + r, e);
  }
}

// colsq[c] = sum over the row blocks, in order, of part[rb * n + c].
__global__ void __launch_bounds__(256) k_sum_blocks(const double* __restrict__ part, int64_t nrb,
                                                    int64_t n, double* __restrict__ colsq) {
  const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (c >= n) return;
  double s = 0.0;
  for (int64_t rb = 0; rb < nrb; ++rb) s += part[rb * n + c];
  colsq[c] = s;
}

__global__ void __launch_bounds__(1024) k_total(const double* __restrict__ v, int64_t count,
                                                double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += 1024) s += v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 32; ++q) t += red[q];
    out[0] = t;
  }
}

__global__ void __launch_bounds__(CHOL_NT) k_chol_inv(const double* __restrict__ S, int b, double tau,
                                                      double* __restrict__ Rinv, int* __restrict__ flags,
                                                      int* __restrict__ dead) {
  chol_inv_cta(S, b, tau, Rinv, flags, dead);
}

__global__ void k_append_rows(const double* __restrict__ Wt, int64_t ldw, int64_t n, int b,
                              double* __restrict__ B, int64_t ldb, int64_t row0,
                              const double* __restrict__ colsum, double p, double* __restrict__ zB) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * b) return;
  const int c = (int)(idx % b);
  const int64_t r = idx / b;
  B[row0 + c + r * ldb] = Wt[r + (int64_t)c * ldw];
  if (zB && r == 0) zB[row0 + c] = p * colsum[c];
}

__global__ void k_fill(double* __restrict__ X, int64_t ld, int64_t rows, int64_t cols, double v) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  X[(idx % rows) + (idx / rows) * ld] = v;
}

cudaError_t col_sums(const double* X, int64_t ld, int64_t rows, int64_t cols, double* sumsq,
                     double* sum, cudaStream_t st) {
  if (cols <= 0) return cudaSuccess;
  k_col_sums<<<(unsigned)cols, 256, 0, st>>>(X, ld, rows, sumsq, sum);
  return launched();
}

int64_t a_stats_part_elems(int64_t m, int64_t n) { return (m + 511) / 512 * n; }

cudaError_t a_stats(const void* A, int dtype, int64_t lda, int64_t m, int64_t n, double* part,
                    double* colsq, int* colE, int* rowE, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(colE, 0, n * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(rowE, 0, m * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int64_t nrb = (m + 511) / 512;
  const dim3 grid((unsigned)nrb, (unsigned)((n + 31) / 32));
  if (dtype == LRA_F32)
    k_a_stats<float><<<grid, 256, 0, st>>>((const float*)A, lda, m, n, part, colE, rowE);
  else
    k_a_stats<double><<<grid, 256, 0, st>>>((const double*)A, lda, m, n, part, colE, rowE);
  e = launched();
  if (e != cudaSuccess) return e;
  k_sum_blocks<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, nrb, n, colsq);
  return launched();
}

cudaError_t total(const double* v, int64_t count, double* out, cudaStream_t st) {
  k_total<<<1, 1024, 0, st>>>(v, count, out);
  return launched();
}

cudaError_t chol_inv(const double* S, int b, double tau, double* Rinv, int* flags, cudaStream_t st,
                     int* dead) {
  k_chol_inv<<<1, CHOL_NT, 0, st>>>(S, b, tau, Rinv, flags, dead);
  return launched();
}

cudaError_t append_rows(const double* Wt, int64_t ldw, int64_t n, int b, double* B, int64_t ldb,
                        int64_t row0, const double* colsum, double p, double* zB, cudaStream_t st) {
  const int64_t total_ = n * b;
  k_append_rows<<<(unsigned)((total_ + 255) / 256), 256, 0, st>>>(Wt, ldw, n, b, B, ldb, row0,
                                                                  colsum, p, zB);
  return launched();
}

cudaError_t fill(double* X, int64_t ld, int64_t rows, int64_t cols, double v, cudaStream_t st) {
  const int64_t total_ = rows * cols;
  if (total_ <= 0) return cudaSuccess;
  k_fill<<<(unsigned)((total_ + 255) / 256), 256, 0, st>>>(X, ld, rows, cols, v);
  return launched();
}

}  // namespace lra
