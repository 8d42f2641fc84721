// Orthonormalisation and reduction kernels of the farPCA block (arxiv
// 2506.03859): the b x b Cholesky factor of a Gram matrix and its inverse (the
// basis Q_j = Y' R^{-1}, the role of Z^{-1} in Alg. 1 step 10), the Frobenius
// norms behind the error indicator (E = ||A||_F^2 - sum_j ||B_j||_F^2, Sec. 2.1),
// and the row append of B_j.  All reductions use a fixed order so repeated runs
// give identical bits.
#include <math.h>

#include <cmath>

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
// SQ = false: the exponents alone (the sums of squares then come from the digit
// cut, which reads A anyway).
template <typename T, bool SQ>
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
      if (SQ) {
        if (k & 1)
          s1 = fma(x, x, s1);
        else
          s0 = fma(x, x, s0);
      }
    }
    double sq = s0 + s1;
    for (int o = 16; o > 0; o >>= 1) {
      if (SQ) sq += __shfl_down_sync(0xffffffffu, sq, o);
      e = max(e, __shfl_down_sync(0xffffffffu, e, o));
    }
    if (lane == 0) {
      if (SQ) part[(int64_t)blockIdx.x * n + c] = sq;
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
                                                      int* __restrict__ dead, int* __restrict__ near) {
  chol_inv_cta(S, b, tau, Rinv, flags, dead, near);
}

// Conversions between FP64 and FP32 by integer operations.  On GB300 a
// conversion instruction runs on the FP64 pipe, which retires about one warp
// instruction per 64 cycles per sub-partition; these run on the integer pipes.
// f64_to_f32: the significand truncated to 24 bits (relative error below 2^-23),
// magnitudes below 2^-126 to zero, above the FP32 range to infinity.
__device__ __forceinline__ float f64_to_f32(double v) {
  const uint64_t u = (uint64_t)__double_as_longlong(v);
  const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((uint32_t)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}
// f32_to_f64: exact for normal values and infinities; FP32 subnormals (below
// 2^-126) to zero.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u, ef = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  if (ef == 0) return __hiloint2double((int)sign, 0);
  const uint32_t ed = ef == 255u ? 2047u : ef - 127u + 1023u;
  return __hiloint2double((int)(sign | (ed << 20) | (m >> 3)), (int)(m << 29));
}

// The FP32 corrections below: a CTA of 128 threads takes NEAR_ROWS = 32 rows;
// warp w computes output columns 16 w .. 16 w + 15 of them (nothing when
// 16 w >= b), lane = row, so that every thread of a warp reads the same entries of
// the small right-hand matrix in shared memory (a broadcast) and its own row's
// entries without bank conflicts.  Many small CTAs keep several warps on every
// sub-partition, which the dependent FMA chains of one warp need.
constexpr int NEAR_THREADS = 128, NEAR_ROWS = 32;

// Thirty-two rows of X (rows x cols, ld ldx, from row r0; columns < 64 read) into
// xs[k][r] as FP32 (f64_to_f32), zero beyond rows and cols: each thread issues its
// 16 loads (consecutive rows across a warp) before converting any.
__device__ __forceinline__ void stage_rows_f32(const double* __restrict__ X, int64_t ldx,
                                               int64_t rows, int64_t cols, int64_t r0,
                                               float (&xs)[64][NEAR_ROWS]) {
  constexpr int PER = 64 * NEAR_ROWS / NEAR_THREADS;
  const int r = threadIdx.x & 31, kb = threadIdx.x >> 5;
  const int64_t i = r0 + r;
  double v[PER];
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int k = kb + 4 * t;
    v[t] = (i < rows && k < cols) ? __ldg(X + i + (int64_t)k * ldx) : 0.0;
  }
#pragma unroll
  for (int t = 0; t < PER; ++t) xs[kb + 4 * t][r] = f64_to_f32(v[t]);
}

// 64 x 64 entries of a column-major matrix (ld ldm, from row k0; rows < kn and
// columns < cn read, zero elsewhere) into ms[k][c] as FP32; with thr, also whether
// any |entry of column c| exceeds the double whose bits are thr[c] (or is a NaN).
// Loads in two batches of 16 per thread.
__device__ __forceinline__ int stage_square_f32(const double* __restrict__ M, int64_t ldm,
                                                int64_t k0, int64_t kn, int cn,
                                                float (&ms)[64][64], const uint64_t* thr) {
  constexpr int PER = 64 * 64 / NEAR_THREADS, BATCH = PER / 2;
  const int c = threadIdx.x & 63, kb = threadIdx.x >> 6;
  const uint64_t th = thr ? thr[c] : ~0ull;
  int big = 0;
#pragma unroll
  for (int h = 0; h < PER; h += BATCH) {
    double v[BATCH];
#pragma unroll
    for (int t = 0; t < BATCH; ++t) {
      const int64_t k = k0 + kb + 2 * (h + t);
      v[t] = (k < kn && c < cn) ? __ldg(M + k + (int64_t)c * ldm) : 0.0;
    }
#pragma unroll
    for (int t = 0; t < BATCH; ++t) {
      big |= ((uint64_t)__double_as_longlong(v[t]) & 0x7FFFFFFFFFFFFFFFull) > th;
      ms[kb + 2 * (h + t)][c] = f64_to_f32(v[t]);
    }
  }
  return big;
}

// acc[c] += sum_{k < kn} xs[k][r] ds[k][c0 + c], c < 16: one load of x and four
// broadcast loads of ds per k, in a short loop (a fully unrolled one overflows the
// instruction cache, and every warp runs it only once).
__device__ __forceinline__ void fma_rows(const float (&xs)[64][NEAR_ROWS], const float (&ds)[64][64],
                                         int kn, int r, int c0, float (&acc)[16]) {
#pragma unroll 4
  for (int k = 0; k < kn; ++k) {
    const float x = xs[k][r];
    const float4* d = reinterpret_cast<const float4*>(&ds[k][c0]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = d[q];
      acc[4 * q] = fmaf(x, v.x, acc[4 * q]);
      acc[4 * q + 1] = fmaf(x, v.y, acc[4 * q + 1]);
      acc[4 * q + 2] = fmaf(x, v.z, acc[4 * q + 2]);
      acc[4 * q + 3] = fmaf(x, v.w, acc[4 * q + 3]);
    }
  }
}

// out = X + X D with D = R^{-1} - I (X: rows x b), when *near is set: the
// Cholesky found every entry of its Gram within 2^-40 of the identity's, so the
// entries of D (the closed form -Phi(S - I)) are within 2^-40 and the correction
// X D needs only FP32: X and D truncated to FP32 (f64_to_f32), products summed in
// FP32, so the correction errs by at most (b + 4) 2^-24 sum_k |X[i, k]| |D[k, c]|;
// the sum, ~2^-40 of X, is added to X in FP64.  Otherwise nothing: the
// FP64-accurate product runs instead.  One FP64 operation per output (the final
// add) and one per diagonal entry of D.
__global__ void __launch_bounds__(NEAR_THREADS) k_rinv_near_identity(
    const double* __restrict__ X, int64_t ldx, int64_t rows, int b, const double* __restrict__ Rinv,
    const int* __restrict__ near, double* __restrict__ out, int64_t ldo) {
  if (__ldcg(near) == 0) return;
  __shared__ __align__(16) float D[64][64];          // D[k][c], zero beyond b
  __shared__ __align__(16) float xs[64][NEAR_ROWS];  // xs[k][r] = X[r0 + r, k]
  const int64_t r0 = (int64_t)blockIdx.x * NEAR_ROWS;
  stage_square_f32(Rinv, b, 0, b, b, D, nullptr);
  stage_rows_f32(X, ldx, rows, b, r0, xs);
  __syncthreads();
  if (threadIdx.x < 64 && threadIdx.x < b) {
    // D's diagonal: R^{-1}_cc - 1, exact in FP64 (R^{-1}_cc near 1)
    const int c = threadIdx.x;
    D[c][c] = f64_to_f32(__ldg(Rinv + c + (int64_t)c * b) - 1.0);
  }
  __syncthreads();
  const int c0 = (threadIdx.x >> 5) * 16, r = threadIdx.x & 31;
  const int64_t i = r0 + r;
  if (i >= rows || c0 >= b) return;
  float acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.0f;
  fma_rows(xs, D, b, r, c0, acc);
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const int cc = c0 + c;
    if (cc < b) out[i + (int64_t)cc * ldo] = __ldg(X + i + (int64_t)cc * ldx) + f32_to_f64(acc[c]);
  }
}

// The second projection of CGS2, Y -= Q F (Q: rows x l, F = Q^T Y: l x b, Y:
// rows x b), in FP32 when F is small enough: every |F[k, c]| within
// g 2^(yE[c] - 1022), where yE[c] is the biased exponent of Y's largest entry in
// column c (so |Y[:, c]| < 2^(yE[c] - 1022)).  With Q and F truncated to FP32
// (f64_to_f32) and the products summed in FP32, the update errs by at most
// (l + 4) 2^-24 sum_k |Q[i, k]| |F[k, c]| <= (l + 4) sqrt(l) 2^-24 max|F[:, c]| (the
// rows of Q have norm <= 1), so with g = 2^-29 / ((l + 4) sqrt(l)) it errs by at
// most 2^-53 2^(yE[c] - 1022), the rounding of Y's largest entries.  After the
// first projection F is of the order of Y's rounding errors, far below that.
// Every CTA stages all of F and takes the same decision (an integer comparison of
// the magnitudes' bits, which a NaN fails); CTA 0 records it in *taken (the
// FP64-accurate update then does nothing); if F is not small, no CTA writes.
// l in chunks of 64.
__global__ void __launch_bounds__(NEAR_THREADS) k_project_fp32(
    const double* __restrict__ Q, int64_t ldq, int64_t rows, int64_t l, const double* __restrict__ F,
    int64_t ldf, int b, const int* __restrict__ yE, double g, double* __restrict__ Y, int64_t ldy,
    int* __restrict__ taken) {
  __shared__ __align__(16) float Fs[64][64];         // Fs[k][c] = F[k0 + k, c], zero beyond l, b
  __shared__ __align__(16) float qs[64][NEAR_ROWS];  // qs[k][r] = Q[r0 + r, k0 + k]
  __shared__ uint64_t thr[64];                       // bits of g 2^(yE[c] - 1022)
  __shared__ int s_big;
  if (threadIdx.x < 64)
    thr[threadIdx.x] = threadIdx.x < b
                           ? (uint64_t)__double_as_longlong(scalbn(g, __ldg(yE + threadIdx.x) - 1022))
                           : 0;
  if (threadIdx.x == 0) s_big = 0;
  const int64_t r0 = (int64_t)blockIdx.x * NEAR_ROWS;
  const int c0 = (threadIdx.x >> 5) * 16, r = threadIdx.x & 31;
  const int64_t i = r0 + r;
  const bool active = i < rows && c0 < b;
  float acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.0f;
  for (int64_t k0 = 0; k0 < l; k0 += 64) {
    __syncthreads();  // thr and s_big set; the previous chunk consumed
    if (stage_square_f32(F, ldf, k0, l, b, Fs, thr)) s_big = 1;
    stage_rows_f32(Q + k0 * ldq, ldq, rows, l - k0, r0, qs);
    __syncthreads();
    if (active) fma_rows(qs, Fs, l - k0 < 64 ? (int)(l - k0) : 64, r, c0, acc);
  }
  __syncthreads();
  const bool small = s_big == 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *taken = small;
  if (!small || !active) return;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const int cc = c0 + c;
    if (cc < b) Y[i + (int64_t)cc * ldy] -= f32_to_f64(acc[c]);
  }
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
  if (!part) {
    if (dtype == LRA_F32)
      k_a_stats<float, false><<<grid, 256, 0, st>>>((const float*)A, lda, m, n, nullptr, colE, rowE);
    else
      k_a_stats<double, false><<<grid, 256, 0, st>>>((const double*)A, lda, m, n, nullptr, colE,
                                                     rowE);
    return launched();
  }
  if (dtype == LRA_F32)
    k_a_stats<float, true><<<grid, 256, 0, st>>>((const float*)A, lda, m, n, part, colE, rowE);
  else
    k_a_stats<double, true><<<grid, 256, 0, st>>>((const double*)A, lda, m, n, part, colE, rowE);
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
                     int* dead, int* near) {
  k_chol_inv<<<1, CHOL_NT, 0, st>>>(S, b, tau, Rinv, flags, dead, near);
  return launched();
}

cudaError_t rinv_near_identity(const double* X, int64_t ldx, int64_t rows, int b, const double* Rinv,
                               const int* near, double* out, int64_t ldo, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if (b <= 0 || b > 64) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)((rows + NEAR_ROWS - 1) / NEAR_ROWS);
  k_rinv_near_identity<<<grid, NEAR_THREADS, 0, st>>>(X, ldx, rows, b, Rinv, near, out, ldo);
  return launched();
}

cudaError_t project_fp32(const double* Q, int64_t ldq, int64_t rows, int64_t l, const double* F,
                         int64_t ldf, int b, const int* yE, double* Y, int64_t ldy, int* taken,
                         cudaStream_t st) {
  if (rows <= 0 || l <= 0) return cudaErrorInvalidValue;
  if (b <= 0 || b > 64) return cudaErrorInvalidValue;
  const double g = std::ldexp(1.0, -29) / (((double)l + 4.0) * std::sqrt((double)l));
  const unsigned grid = (unsigned)((rows + NEAR_ROWS - 1) / NEAR_ROWS);
  k_project_fp32<<<grid, NEAR_THREADS, 0, st>>>(Q, ldq, rows, l, F, ldf, b, yE, g, Y, ldy, taken);
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
