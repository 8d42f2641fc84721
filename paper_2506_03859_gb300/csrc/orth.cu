// Orthonormalisation and reduction kernels of the farPCA block (arxiv
// 2506.03859): the b x b Cholesky factor of a Gram matrix and its inverse (the
// basis Q_j = Y' R^{-1}, the role of Z^{-1} in Alg. 1 step 10), the Frobenius
// norms behind the error indicator (E = ||A||_F^2 - sum_j ||B_j||_F^2, Sec. 2.1),
// and the row append of B_j.  All reductions use a fixed order so repeated runs
// give identical bits.
#include <math.h>

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

// Upper Cholesky R of S (b <= 64) and R^{-1}, right-looking: at column c the
// pivot d = S_cc - sum_{k<c} R_kc^2 (the trailing block already holds the
// subtracted sum) must pass d > tau * S_cc (original diagonal) and be finite;
// with r = 1/sqrt(d), R_cc = d r and row c of R is the pivot row times r; the
// trailing block loses the outer product of that row.  R^{-1} comes out of the
// same sweep as Z^T, Z = L^{-1} for L = R^T by forward substitution: once row c
// of R (column c of L) and r are known, row c of Z is row c of the reduced
// right-hand side (the identity at the start) times r, and every row i > c of
// the right-hand side loses R_ci times it.  Both updates are one FMA per
// element; Z is lower triangular, so only columns <= c change.
//
// On GB300 one dependent FP64 operation takes ~64 cycles and the SM's FP64 pipe
// retires about one warp instruction per ~19 cycles, so the sweep is laid out
// around the chain of pivots: while the other 31 warps apply column c's updates
// (about one element each, so that the index arithmetic and shared-memory
// latencies of an update overlap across warps instead of queueing in a few),
// thread 0 already finishes pivot c + 1 (its last update, the test and the
// reciprocal square root).  Two barriers per column.  The trailing pairs
// (i, j), c < i <= j, come from a table of all pairs i <= j sorted by i
// descending (those of column c are its first (b-1-c)(b-c)/2 entries); the Z
// updates (i > c, j <= c) are numbered densely, i = c + 1 + f div (c + 1).
//
// Near the identity the sweep is not needed.  The second Gram of CholQR2 is
// S = I + E with E of the order of the first pass's loss of orthogonality.
// With R = I + U (U upper), R^T R = I + E gives U = Phi(E) - Phi(U^T U), where
// Phi keeps the strict upper triangle and halves the diagonal, and
// R^{-1} = I - U + U^2 - ...; so R^{-1} = I - Phi(E) up to terms bounded by
// 2 b max|E|^2 per entry.  When max|E| <= 2^-34 that is at most 2^-61 for
// b <= 64, below the rounding of the entries near 1 and far below what
// X R^{-1} can resolve, and R^{-1} is written directly (every pivot is then
// ~1 and passes the breakdown test).
constexpr int CHOL_NT = 1024;
constexpr double CHOL_NEAR_I = 0x1p-34;

//
// Skip mode (dead != NULL, the first pass over a power-step panel): a failed
// pivot marks column c dependent instead of ending the factorisation.  Its
// reciprocal pivot is taken as 0, so row c of R beyond the diagonal and row c of
// Z are zero: the column updates nothing after it, no other column of R^{-1}
// refers to it, and column c of R^{-1} is zero (the caller replaces that column
// of X R^{-1}).
__global__ void __launch_bounds__(CHOL_NT) k_chol_inv(const double* __restrict__ S, int b, double tau,
                                                      double* __restrict__ Rinv, int* __restrict__ flags,
                                                      int* __restrict__ dead) {
  constexpr int NWORK = CHOL_NT - 32;
  __shared__ double M[64][65];  // trailing block (upper triangle); row c becomes row c of R
  __shared__ double Z[64][65];  // right-hand side, rows of Z once final (lower triangle)
  __shared__ double Sd[64], dpiv[64], rpiv[64];
  __shared__ uint16_t pairs[64 * 65 / 2];  // (i << 8) | j, i <= j, i descending
  __shared__ int bad;
  __shared__ int sdead[64];
  const int t = threadIdx.x;
  const bool skip = dead != nullptr;
  // workers: warps 1 .. 31; thread 0 takes the pivots
  const int wk = t - 32;
  int far = 0;  // an entry of S - I above 2^-34, or not finite
  for (int e = t; e < b * b; e += CHOL_NT) {
    const int i = e % b, j = e / b;
    const double v = S[i + j * b];
    M[i][j] = v;
    Z[i][j] = (i == j) ? 1.0 : 0.0;
    far |= !(fabs(i == j ? v - 1.0 : v) <= CHOL_NEAR_I);
  }
  if (!__syncthreads_or(far)) {
    // R^{-1} = I - Phi(S - I): -S_ij above the diagonal, 1 - (S_ii - 1)/2 on it
    for (int e = t; e < b * b; e += CHOL_NT) {
      const int i = e % b, j = e / b;
      const double v = M[i][j];
      Rinv[i + j * b] = i < j ? -v : (i == j ? fma(-0.5, v - 1.0, 1.0) : 0.0);
    }
    if (skip && t < b) dead[t] = 0;
    return;
  }
  if (t < 64) sdead[t] = 0;
  // entry e of the pair table: rows b-1, b-2, ... in turn, row i holding j = i..b-1;
  // the rows above i (i' > i) take sum_{i' > i} (b - i') = (b-1-i)(b-i)/2 entries
  for (int i = t; i < b; i += CHOL_NT) {
    const int base = (b - 1 - i) * (b - i) / 2;
    for (int j = i; j < b; ++j) pairs[base + (j - i)] = (uint16_t)((i << 8) | j);
  }
  if (t < b) Sd[t] = S[t + t * b];
  if (t == 0) {
    const double d = S[0];
    const int fail = !(isfinite(d) && d > tau * d);
    bad = fail && !skip;
    if (fail && skip) sdead[0] = 1;
    dpiv[0] = d;
    rpiv[0] = fail ? 0.0 : rsqrt(d);
  }
  __syncthreads();
  for (int c = 0; c < b; ++c) {
    if (bad) break;  // set before the last barrier: the same decision in every thread
    const double r = rpiv[c];
    // row c of R (R_cc = d r) and row c of Z (both zero for a dependent column)
    if (t >= c && t < b) M[c][t] = (r == 0.0) ? 0.0 : (t == c) ? dpiv[c] * r : M[c][t] * r;
    else if (t >= 64 && t - 64 <= c) Z[c][t - 64] = (r == 0.0) ? 0.0 : Z[c][t - 64] * r;
    __syncthreads();
    const int nt = b - c - 1;
    if (t == 0) {
      if (nt > 0) {
        const double rc1 = M[c][c + 1];
        const double d = fma(-rc1, rc1, M[c + 1][c + 1]);
        if (!(isfinite(d) && d > tau * Sd[c + 1])) {
          if (skip) {
            sdead[c + 1] = 1;
            dpiv[c + 1] = 0.0;
            rpiv[c + 1] = 0.0;
          } else {
            bad = 1;
          }
        } else {
          dpiv[c + 1] = d;
          rpiv[c + 1] = rsqrt(d);
        }
      }
    } else if (wk >= 0) {
      const int ntrail = nt * (nt + 1) / 2, ntot = ntrail + nt * (c + 1);
      const float kinv = 1.0f / (float)(c + 1);
      for (int e = wk; e < ntot; e += NWORK) {
        if (e < ntrail) {
          const int ij = pairs[e], i = ij >> 8, j = ij & 255;
          if (i != c + 1 || j != c + 1) M[i][j] = fma(-M[c][i], M[c][j], M[i][j]);  // pivot: thread 0
        } else {
          const int f = e - ntrail;
          const int q = (int)(((float)f + 0.5f) * kinv);  // f div (c + 1); f < 4096, exact enough
          const int j = f - q * (c + 1), i = c + 1 + q;
          Z[i][j] = fma(-M[c][i], Z[c][j], Z[i][j]);
        }
      }
    }
    __syncthreads();
  }
  if (bad) {
    if (t == 0) atomicOr(flags, FLAG_BREAKDOWN);
    for (int e = t; e < b * b; e += CHOL_NT) Rinv[e] = 0.0;
    return;
  }
  // R^{-1} = Z^T
  for (int e = t; e < b * b; e += CHOL_NT) {
    const int i = e % b, j = e / b;
    Rinv[i + j * b] = i <= j ? Z[j][i] : 0.0;
  }
  if (skip && t < b) dead[t] = sdead[t];
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
