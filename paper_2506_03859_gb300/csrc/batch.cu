// Batched form: thousands of independent fixed-precision farPCA problems
// (arxiv 2506.03859 Alg. 1 in the QB form of Sec. 2.1, Omega the fixed-zeta
// sparse sign matrix) advanced together, one block per step, by one CUDA graph
// whose body is a block step and which repeats it on the device (a conditional
// while node) until no problem is active.
//
// Every kernel of a step works on all active problems at once, over a static
// list of (problem, chunk) tiles ordered by problem size, so the hardware
// scheduler balances uneven sizes.  Data and passes are FP32 (the FP32 form of
// the workload): A is FP32, the products with A and with Q accumulate in FP32;
// Gram matrices are summed in FP64 from FP32 partials of at most 64 terms, the
// Cholesky factors, ||A||_F^2 and the indicator are FP64.  The orthonormal basis
// (the Q factor of QR with positive diagonal R, as in the FP64 path) comes from
// shifted Cholesky QR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa,
// SIAM J. Sci. Comput. 42 (2020)): a Cholesky QR of the Gram shifted by
// 2^-16 tr(X^T X) (four times the bound 64 2^-24 tr on the rounding of the FP32
// Gram partials, so the shifted Gram stays positive definite), then two plain
// ones; this keeps condition numbers up to ~1e6 stable in FP32.
// The power step is taken in its stabilised form: the deflated W of Alg. 1,
// A^T S0 - B^T (B Omega_j) = A^T (I - Q Q^T) A Omega_j, is formed as A^T Q0 with
// Q0 = orth((I - Q Q^T) A Omega_j) (classical Gram-Schmidt, twice).  A^T Q0 =
// W R0^{-1} has W's span and the same Q factor G, with condition number
// ~sigma_1 / sigma_b instead of its square.  A block breaks down when a diagonal
// entry of R = R3 R2 R1 of the sketch or of Y' is not above 2^-20 (16 times
// FP32's rounding) times its column's norm; W' is not tested (a rank-deficient
// A breaks down at Y' = A G).  The FP64 path tests its Gram pivots against
// 1e-13 S_cc.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.cuh"
#include "batch_plan.h"
#include "philox.cuh"

namespace lra {
namespace {

constexpr double BATCH_TAU = 0x1p-20;
constexpr int ZMAX = 16;  // largest zeta of the batched form

struct BProb {
  const float* A;
  int64_t lda;
  int m, n, cap, lmax, zeta;
  double eps2;
  uint32_t k0, k1;
  float *Q, *Bt, *X, *W, *F, *Rinv, *omv;
  int* omr;
  double *rdiag, *cnorm;
  int c32_first, c32_count;    // this problem's tiles in the 32-column list (||A||^2)
  int g64_first, g64_count;    // its 64-column groups (partial sums of ||B_j||_F^2)
  // state
  double normA2, E;
  int status, rank, active, broke;
};

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
  return s;  // thread 0
}

// ||A_i||_F^2 partials: tile (problem, 32 columns); warp w, columns 4w..4w+3.
__global__ void __launch_bounds__(256) k_b_norm(const BProb* __restrict__ pr,
                                                const int2* __restrict__ tiles,
                                                double* __restrict__ part) {
  __shared__ double red[8];
  const int2 t = tiles[blockIdx.x];
  const BProb& p = pr[t.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0.0;
  for (int q = 0; q < 4; ++q) {
    const int c = t.y + warp * 4 + q;
    if (c >= p.n) break;
    const float* col = p.A + (int64_t)c * p.lda;
    float acc = 0.f;  // at most 64 terms
    for (int i = lane; i < p.m; i += 32) acc = fmaf(col[i], col[i], acc);
    s += (double)acc;
  }
  const double tot = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_b_start(BProb* __restrict__ pr, int np, const double* __restrict__ part,
                          int* __restrict__ jp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *jp = 0;
  if (i >= np) return;
  BProb& p = pr[i];
  double s = 0.0;
  for (int q = 0; q < p.c32_count; ++q) s += part[p.c32_first + q];
  p.normA2 = s;
  p.E = s;
  p.rank = 0;
  p.broke = 0;
  if (!isfinite(s)) {
    p.status = LRA_ERR_INVALID_ARG;
    p.active = 0;
  } else if (s == 0.0) {
    p.status = LRA_OK;
    p.active = 0;
  } else {
    p.status = LRA_NOT_CONVERGED;
    p.active = 1;
  }
}

// Omega_j of problem i: column c draws rows until zeta distinct ones are
// accepted (the fixed-zeta sparse sign generator of the single-matrix path).
template <int B>
__global__ void k_b_omega(BProb* __restrict__ pr, int np, const int* __restrict__ jp) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= np * B) return;
  BProb& p = pr[g / B];
  if (!p.active) return;
  const uint32_t j = (uint32_t)*jp, c = (uint32_t)(g % B);
  const float v = 1.0f / sqrtf((float)p.zeta);
  int taken[ZMAX];
  int cnt = 0;
  const int max_draws = 64 * p.zeta + 1024;
  for (int t = 0; t < max_draws && cnt < p.zeta; ++t) {
    const U32x4 u = philox4x32_10((uint32_t)t, j, c, TAG_SPARSE_SIGN, p.k0, p.k1);
    const int r = (int)(((uint64_t)u.x * (uint64_t)p.n) >> 32);
    bool dup = false;
    for (int q = 0; q < cnt; ++q) dup |= (taken[q] == r);
    if (dup) continue;
    taken[cnt] = r;
    p.omr[c * ZMAX + cnt] = r;
    p.omv[c * ZMAX + cnt] = (u.y & 1u) ? -v : v;
    ++cnt;
  }
  if (cnt < p.zeta) p.broke = 1;
}

// X = A Omega_j: tile (problem, 128 rows), a thread per row.
template <int B>
__global__ void __launch_bounds__(128) k_b_sketch(const BProb* __restrict__ pr,
                                                  const int2* __restrict__ tiles) {
  __shared__ int sr[B * ZMAX];
  __shared__ float sv[B * ZMAX];
  const int2 t = tiles[blockIdx.x];
  const BProb& p = pr[t.x];
  if (!p.active || p.broke) return;
  const int z = p.zeta;
  for (int e = threadIdx.x; e < B * ZMAX; e += 128) {
    const bool in = (e % ZMAX) < z;
    sr[e] = in ? p.omr[e] : 0;
    sv[e] = in ? p.omv[e] : 0.f;
  }
  __syncthreads();
  const int i = t.y + threadIdx.x;
  if (i >= p.m) return;
  for (int c = 0; c < B; ++c) {
    float acc = 0.f;
    for (int q = 0; q < z; ++q) acc = fmaf(sv[c * ZMAX + q], p.A[i + (int64_t)sr[c * ZMAX + q] * p.lda], acc);
    p.X[i + (int64_t)c * p.m] = acc;
  }
}

enum TnMode { TN_ATX = 0, TN_QTY = 1, TN_QTA = 2 };

// C = X^T Y over a tile of 64 CPT columns of X, 64 threads, each thread CPT
// columns (c, c + 64, ...; CPT = the problem's tn, its class's tile shape): the
// thread streams its columns down the rows (16-byte loads where a column is
// aligned) while the 64-row chunk of Y (b columns) sits in shared memory, read by
// all threads at the same address, each value used for all CPT columns; each
// thread keeps its CPT b sums in registers.  A column's sum runs over the rows in
// the same order whatever CPT is.
//   TN_ATX: W = A^T X (n x b);  TN_QTY: F = Q^T X (l x b);
//   TN_QTA: B_j^T = A^T Q_j into Bt's columns l.., and sum of squares -> part.
template <int B, int MODE, int CPT>
__device__ __forceinline__ void tn_tile(const BProb& p, int2 t, int l, int cols, double* __restrict__ part,
                                        float (*ys)[B], double* red) {
  const float* X = MODE == TN_QTY ? p.Q : p.A;
  const int64_t ldx = MODE == TN_QTY ? (int64_t)p.m : p.lda;
  const float* Y = MODE == TN_QTA ? p.Q + (int64_t)l * p.m : p.X;
  int c[CPT];
  bool mine[CPT];
  const float* col[CPT];
  bool vec = true;
#pragma unroll
  for (int h = 0; h < CPT; ++h) {
    c[h] = t.y + threadIdx.x + 64 * h;
    mine[h] = c[h] < cols;
    col[h] = X + (int64_t)(mine[h] ? c[h] : t.y) * ldx;
    vec = vec && ((reinterpret_cast<uintptr_t>(col[h]) & 15) == 0);
  }
  float acc[CPT][B];
#pragma unroll
  for (int h = 0; h < CPT; ++h)
#pragma unroll
    for (int k = 0; k < B; ++k) acc[h][k] = 0.f;
  for (int r0 = 0; r0 < p.m; r0 += 64) {
    const int rn = min(64, p.m - r0);
    for (int e = threadIdx.x; e < 64 * B; e += 64) {
      const int rr = e % 64, k = e / 64;
      ys[rr][k] = rr < rn ? Y[(r0 + rr) + (int64_t)k * p.m] : 0.f;
    }
    __syncthreads();
    if (vec && rn == 64) {
#pragma unroll
      for (int q0 = 0; q0 < 16; q0 += 4) {
        float4 a4[CPT][4];
#pragma unroll
        for (int h = 0; h < CPT; ++h)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            a4[h][q] = __ldg(reinterpret_cast<const float4*>(col[h] + r0 + 4 * (q0 + q)));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int rr = 4 * (q0 + q) + e;
#pragma unroll
            for (int k = 0; k < B; k += 4) {
              const float4 y = *reinterpret_cast<const float4*>(&ys[rr][k]);
#pragma unroll
              for (int h = 0; h < CPT; ++h) {
                const float ah = e == 0 ? a4[h][q].x : e == 1 ? a4[h][q].y : e == 2 ? a4[h][q].z : a4[h][q].w;
                acc[h][k] = fmaf(ah, y.x, acc[h][k]);
                acc[h][k + 1] = fmaf(ah, y.y, acc[h][k + 1]);
                acc[h][k + 2] = fmaf(ah, y.z, acc[h][k + 2]);
                acc[h][k + 3] = fmaf(ah, y.w, acc[h][k + 3]);
              }
            }
          }
        }
      }
    } else {
      for (int rr = 0; rr < rn; ++rr) {
#pragma unroll
        for (int h = 0; h < CPT; ++h) {
          const float ah = col[h][r0 + rr];
#pragma unroll
          for (int k = 0; k < B; ++k) acc[h][k] = fmaf(ah, ys[rr][k], acc[h][k]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int h = 0; h < CPT; ++h) {
    double sq = 0.0;  // this thread's column of the 64-column group t.y / 64 + h
    if (mine[h]) {
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const float v = acc[h][k];
        if (MODE == TN_ATX) p.W[c[h] + (int64_t)k * p.n] = v;
        if (MODE == TN_QTY) p.F[c[h] + (int64_t)k * p.lmax] = v;
        if (MODE == TN_QTA) {
          p.Bt[c[h] + (int64_t)(l + k) * p.n] = v;
          sq += (double)v * (double)v;
        }
      }
    }
    if (MODE == TN_QTA) {
      // one partial per 64-column group, summed in the same order whatever the tile
      const double s2 = block_sum(sq, red);
      const int g = t.y / 64 + h;
      if (threadIdx.x == 0 && g < p.g64_count) part[p.g64_first + g] = s2;
    }
  }
}

// One shape class's tiles: tiles[off ..] (TN_QTA: the partial sums of the tile's
// 64-column groups in part[g64_first + group]).
template <int B, int MODE, int CPT>
__global__ void __launch_bounds__(64) k_b_tn(const BProb* __restrict__ pr,
                                             const int2* __restrict__ tiles, int off,
                                             const int* __restrict__ jp,
                                             double* __restrict__ part) {
  __shared__ __align__(16) float ys[64][B];
  __shared__ double red[2];
  const int2 t = tiles[off + (int)blockIdx.x];
  const BProb& p = pr[t.x];
  const int l = *jp * B;
  const bool live = p.active && !p.broke;
  const int cols = MODE == TN_QTY ? l : p.n;
  if (!live || t.y >= cols) {
    if (MODE == TN_QTA && threadIdx.x == 0)
      for (int h = 0; h < CPT; ++h)
        if (t.y / 64 + h < p.g64_count) part[p.g64_first + t.y / 64 + h] = 0.0;
    return;
  }
  tn_tile<B, MODE, CPT>(p, t, l, cols, part, ys, red);
}

enum NnMode { NN_AX = 0, NN_YQF = 1 };

// Row tile (problem, 64 RPT rows), 64 threads, each thread RPT rows i, i + 64, ...
// (RPT = the problem's nn, its class's tile shape):
//   NN_AX: X = A W (m x b, W = G after orthonormalisation);  NN_YQF: X -= Q F.
// The 64-column chunk of the right operand sits in shared memory, each value used
// for all RPT rows.  A row's sum runs over the columns in the same order whatever
// RPT is.
template <int B, int MODE, int RPT>
__device__ __forceinline__ void nn_tile(const BProb& p, int2 t, int K, float (*ys)[B]) {
  const float* X = MODE == NN_AX ? p.A : p.Q;
  const int64_t ldx = MODE == NN_AX ? p.lda : (int64_t)p.m;
  const float* Y = MODE == NN_AX ? p.W : p.F;
  const int64_t ldy = MODE == NN_AX ? (int64_t)p.n : (int64_t)p.lmax;
  int i[RPT];
  bool in[RPT];
  const float* x[RPT];
#pragma unroll
  for (int h = 0; h < RPT; ++h) {
    i[h] = t.y + threadIdx.x + 64 * h;
    in[h] = i[h] < p.m;
    x[h] = X + (in[h] ? i[h] : 0);
  }
  float acc[RPT][B];
#pragma unroll
  for (int h = 0; h < RPT; ++h)
#pragma unroll
    for (int k = 0; k < B; ++k) acc[h][k] = 0.f;
  for (int k0 = 0; k0 < K; k0 += 64) {
    const int kn = min(64, K - k0);
    for (int e = threadIdx.x; e < 64 * B; e += 64) {
      const int kk = e % 64, k = e / 64;
      ys[kk][k] = kk < kn ? Y[(k0 + kk) + (int64_t)k * ldy] : 0.f;
    }
    __syncthreads();
    int kk = 0;
    // eight columns' loads for every row in flight, then their FMAs
    for (; kk + 8 <= kn; kk += 8) {
      float a[RPT][8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int h = 0; h < RPT; ++h) a[h][u] = __ldg(x[h] + (int64_t)(k0 + kk + u) * ldx);
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int k = 0; k < B; k += 4) {
          const float4 y = *reinterpret_cast<const float4*>(&ys[kk + u][k]);
#pragma unroll
          for (int h = 0; h < RPT; ++h) {
            acc[h][k] = fmaf(a[h][u], y.x, acc[h][k]);
            acc[h][k + 1] = fmaf(a[h][u], y.y, acc[h][k + 1]);
            acc[h][k + 2] = fmaf(a[h][u], y.z, acc[h][k + 2]);
            acc[h][k + 3] = fmaf(a[h][u], y.w, acc[h][k + 3]);
          }
        }
    }
    for (; kk < kn; ++kk) {
#pragma unroll
      for (int h = 0; h < RPT; ++h) {
        const float ah = x[h][(int64_t)(k0 + kk) * ldx];
#pragma unroll
        for (int k = 0; k < B; ++k) acc[h][k] = fmaf(ah, ys[kk][k], acc[h][k]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int h = 0; h < RPT; ++h) {
    if (!in[h]) continue;
#pragma unroll
    for (int k = 0; k < B; ++k) {
      float* o = p.X + i[h] + (int64_t)k * p.m;
      if (MODE == NN_AX)
        *o = acc[h][k];
      else
        *o -= acc[h][k];
    }
  }
}

// One shape class's tiles: tiles[off ..].
template <int B, int MODE, int RPT>
__global__ void __launch_bounds__(64) k_b_nn(const BProb* __restrict__ pr,
                                             const int2* __restrict__ tiles, int off,
                                             const int* __restrict__ jp) {
  __shared__ __align__(16) float ys[64][B];
  const int2 t = tiles[off + (int)blockIdx.x];
  const BProb& p = pr[t.x];
  if (!p.active || p.broke) return;
  const int l = *jp * B;
  const int K = MODE == NN_AX ? p.n : l;
  if (K == 0) return;
  nn_tile<B, MODE, RPT>(p, t, K, ys);
}

// One pass of shifted Cholesky QR3 on the rows x b panel (W: rows n, else X:
// rows m) of each problem, one CTA per problem: the Gram in FP64 from FP32
// partials over 64 rows, then (warp 0) the Cholesky factor R (FP64) and R^{-1}
// (stored FP32).  pass 0 adds the shift and records the column norms; pass 2
// tests diag(R3 R2 R1) for breakdown.
template <int B, bool ON_W>
__global__ void __launch_bounds__(256) k_b_gram_chol(BProb* __restrict__ pr, int pass) {
  constexpr int NE = (B * B + 255) / 256;
  __shared__ float xc[64][B + 1];
  __shared__ double gs[B][B + 1];
  __shared__ double rs[B][B + 1];
  __shared__ double ri[B][B + 1];
  __shared__ int s_bad;
  BProb& p = pr[blockIdx.x];
  if (!p.active || p.broke) return;
  const int rows = ON_W ? p.n : p.m;
  const float* X = ON_W ? p.W : p.X;
  double g[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) g[q] = 0.0;
  for (int r0 = 0; r0 < rows; r0 += 64) {
    for (int e = threadIdx.x; e < 64 * B; e += 256) {
      const int rr = e % 64, k = e / 64;
      xc[rr][k] = (r0 + rr < rows) ? X[(r0 + rr) + (int64_t)k * rows] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NE; ++q) {
      const int e = threadIdx.x + 256 * q;
      if (e < B * B) {
        const int a = e / B, b2 = e % B;
        float s = 0.f;
        for (int rr = 0; rr < 64; ++rr) s = fmaf(xc[rr][a], xc[rr][b2], s);
        g[q] += (double)s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = threadIdx.x + 256 * q;
    if (e < B * B) gs[e / B][e % B] = g[q];
  }
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  if (pass == 0) {
    double tr = 0.0;
    for (int k = 0; k < B; ++k) tr += gs[k][k];
    const double shift = 0x1p-16 * tr;
    __syncwarp();
    if (lane < B) {
      p.cnorm[lane] = sqrt(gs[lane][lane]);
      p.rdiag[lane] = 1.0;
      gs[lane][lane] += shift;
    }
    __syncwarp();
  }
  // right-looking Cholesky, lanes over the columns q: R[c][q] for q >= c
  for (int c = 0; c < B; ++c) {
    const double d = gs[c][c];
    const bool ok = isfinite(d) && d > 0.0;
    if (!ok) {
      if (lane == 0) s_bad = 1;
      break;
    }
    const double rcc = sqrt(d);
    if (lane >= c && lane < B) rs[c][lane] = lane == c ? rcc : gs[c][lane] / rcc;
    __syncwarp();
    if (lane > c && lane < B)
      for (int a = c + 1; a <= lane; ++a) gs[a][lane] -= rs[c][a] * rs[c][lane];
    __syncwarp();
  }
  __syncwarp();
  if (s_bad) {
    if (lane == 0) p.broke = 1;
    return;
  }
  // R^{-1} (upper), lanes over its columns k
  if (lane < B) {
    for (int a = 0; a < B; ++a) ri[a][lane] = 0.0;
    ri[lane][lane] = 1.0 / rs[lane][lane];
    for (int a = lane - 1; a >= 0; --a) {
      double s = 0.0;
      for (int u = a + 1; u <= lane; ++u) s += rs[a][u] * ri[u][lane];
      ri[a][lane] = -s / rs[a][a];
    }
  }
  __syncwarp();
  if (lane < B) {
    for (int a = 0; a < B; ++a) p.Rinv[a * B + lane] = (float)ri[a][lane];
    p.rdiag[lane] *= rs[lane][lane];
  }
  __syncwarp();
  const bool bad = !ON_W && pass == 2 && lane < B && !(p.rdiag[lane] > BATCH_TAU * p.cnorm[lane]);
  if (__any_sync(0xffffffffu, bad) && lane == 0) p.broke = 1;
}

// panel <- panel R^{-1} for a tile (problem, 128 rows); TO_Q: the result goes to
// Q's columns l.. (the last pass of the basis step).
template <int B, bool ON_W, bool TO_Q>
__global__ void __launch_bounds__(128) k_b_rinv(const BProb* __restrict__ pr,
                                                const int2* __restrict__ tiles,
                                                const int* __restrict__ jp) {
  __shared__ float rv[B][B];
  const int2 t = tiles[blockIdx.x];
  const BProb& p = pr[t.x];
  if (!p.active || p.broke) return;
  for (int e = threadIdx.x; e < B * B; e += 128) rv[e / B][e % B] = p.Rinv[e];
  __syncthreads();
  const int rows = ON_W ? p.n : p.m;
  const int i = t.y + threadIdx.x;
  if (i >= rows) return;
  float* X = ON_W ? p.W : p.X;
  float x[B];
#pragma unroll
  for (int k = 0; k < B; ++k) x[k] = X[i + (int64_t)k * rows];
  float* out = TO_Q ? p.Q + (int64_t)(*jp * B) * p.m : X;
#pragma unroll
  for (int k = 0; k < B; ++k) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a <= k; ++a) s = fmaf(x[a], rv[a][k], s);
    out[i + (int64_t)k * rows] = s;
  }
}

// E -= ||B_j||_F^2 (the tile partials, in order); stop test; count the
// problems still active.
template <int B>
__global__ void k_b_indicator(BProb* __restrict__ pr, int np, const int* __restrict__ jp,
                              const double* __restrict__ part, int* __restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  BProb& p = pr[i];
  if (!p.active) return;
  const int j = *jp;
  if (p.broke) {
    p.status = LRA_BREAKDOWN;
    p.active = 0;
    p.broke = 0;
    return;
  }
  double s = 0.0;
  for (int q = 0; q < p.g64_count; ++q) s += part[p.g64_first + q];
  p.E -= s;
  p.rank = (j + 1) * B;
  if (p.E < p.eps2 * p.normA2) {
    p.status = LRA_OK;
    p.active = 0;
  } else if (j + 1 >= p.cap) {
    p.status = LRA_NOT_CONVERGED;
    p.active = 0;
  } else {
    atomicAdd(count, 1);
  }
}

// End of a step: j += 1, and the while node repeats while a problem is active
// (graph mode); without the graph, *more tells the host.
template <bool GRAPH>
__global__ void k_b_next(int* __restrict__ jp, int* __restrict__ count, int max_steps,
                         cudaGraphConditionalHandle h, int* __restrict__ more_out) {
  const int j = *jp + 1;
  *jp = j;
  const int more = (*count > 0) && (j < max_steps);
  *count = 0;
  if (GRAPH)
    cudaGraphSetConditional(h, more ? 1u : 0u);
  else
    *more_out = more;
}

}  // namespace
}  // namespace lra

struct lra_batch {
  int np = 0, b = 0, P = 0, max_steps = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  lra::BProb* d_pr = nullptr;
  std::vector<lra::BProb> h_pr;  // after lra_batch_run: the final state
  std::vector<int> order;        // caller index -> internal index
  int2 *d_c32 = nullptr, *d_ctn = nullptr, *d_rm = nullptr, *d_rn = nullptr, *d_qtn = nullptr,
       *d_rnn = nullptr;
  int n_c32 = 0, n_rm = 0, n_rn = 0;
  int ctn_off[4] = {}, qtn_off[4] = {}, rnn_off[4] = {};  // the tunable lists' class sections
  // the tile shape in use, and what re-planning for another one needs
  lra::BatchTiling tiling = lra::batch_default_tiling();
  std::vector<int64_t> ms, ns;
  int max_blocks = 0;
  std::vector<lra::BProb> h_init;  // the problems as created (pointers, parameters, shapes)
  double* d_part = nullptr;
  int *d_j = nullptr, *d_count = nullptr, *d_more = nullptr;
  bool graph_mode = true;
  char* d_pool = nullptr;
  int64_t pool_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t launches_per_step = 0;
  int steps_last = 0;
};

namespace lra {
namespace {

// The X^T Y and row products: one launch per shape class present, each with the
// kernel of its class's tile shape.
template <int B, int MODE, typename F>
void tn_launch(lra_batch* bt, const int2* tiles, const int* off, F&& L) {
  for (int c = 0; c < BATCH_CLASSES; ++c) {
    const int cnt = off[c + 1] - off[c];
    if (cnt <= 0) continue;
    const int v = bt->tiling.tn[c];
    if (v == 1)
      k_b_tn<B, MODE, 1><<<cnt, 64, 0, bt->st>>>(bt->d_pr, tiles, off[c], bt->d_j, bt->d_part);
    else if (v == 4)
      k_b_tn<B, MODE, 4><<<cnt, 64, 0, bt->st>>>(bt->d_pr, tiles, off[c], bt->d_j, bt->d_part);
    else
      k_b_tn<B, MODE, 2><<<cnt, 64, 0, bt->st>>>(bt->d_pr, tiles, off[c], bt->d_j, bt->d_part);
    L(cudaGetLastError());
  }
}

template <int B, int MODE, typename F>
void nn_launch(lra_batch* bt, F&& L) {
  for (int c = 0; c < BATCH_CLASSES; ++c) {
    const int cnt = bt->rnn_off[c + 1] - bt->rnn_off[c];
    if (cnt <= 0) continue;
    const int v = bt->tiling.nn[c];
    if (v == 1)
      k_b_nn<B, MODE, 1><<<cnt, 64, 0, bt->st>>>(bt->d_pr, bt->d_rnn, bt->rnn_off[c], bt->d_j);
    else if (v == 4)
      k_b_nn<B, MODE, 4><<<cnt, 64, 0, bt->st>>>(bt->d_pr, bt->d_rnn, bt->rnn_off[c], bt->d_j);
    else
      k_b_nn<B, MODE, 2><<<cnt, 64, 0, bt->st>>>(bt->d_pr, bt->d_rnn, bt->rnn_off[c], bt->d_j);
    L(cudaGetLastError());
  }
}

// The kernels of one block step, on bt->st (captured into the graph's body, or
// launched directly when the batch runs without the graph).
template <int B>
cudaError_t issue_step(lra_batch* bt, bool graph, cudaGraphConditionalHandle h) {
  cudaStream_t st = bt->st;
  const int np = bt->np;
  uint64_t n = 0;
  cudaError_t first = cudaSuccess;
  auto L = [&](cudaError_t le) {
    ++n;
    if (first == cudaSuccess) first = le;
  };
  BProb* pr = bt->d_pr;
  const int* jp = bt->d_j;
  k_b_omega<B><<<(np * B + 127) / 128, 128, 0, st>>>(pr, np, jp);
  L(cudaGetLastError());
  k_b_sketch<B><<<bt->n_rm, 128, 0, st>>>(pr, bt->d_rm);
  L(cudaGetLastError());
  // X <- (I - Q Q^T) X, twice; then X <- orth(X) (into Q's columns l.. when to_q)
  auto project = [&]() {
    for (int pass = 0; pass < 2; ++pass) {
      tn_launch<B, TN_QTY>(bt, bt->d_qtn, bt->qtn_off, L);
      nn_launch<B, NN_YQF>(bt, L);
    }
  };
  auto orth_x = [&](bool to_q) {
    for (int ps = 0; ps < 3; ++ps) {
      k_b_gram_chol<B, false><<<np, 256, 0, st>>>(pr, ps);
      L(cudaGetLastError());
      if (ps == 2 && to_q)
        k_b_rinv<B, false, true><<<bt->n_rm, 128, 0, st>>>(pr, bt->d_rm, jp);
      else
        k_b_rinv<B, false, false><<<bt->n_rm, 128, 0, st>>>(pr, bt->d_rm, jp);
      L(cudaGetLastError());
    }
  };
  if (bt->P >= 1) {
    // W' = A^T orth((I - Q Q^T) A Omega_j); G = orth(W'); Y_j = A G
    project();
    orth_x(false);
    tn_launch<B, TN_ATX>(bt, bt->d_ctn, bt->ctn_off, L);
    for (int ps = 0; ps < 3; ++ps) {
      k_b_gram_chol<B, true><<<np, 256, 0, st>>>(pr, ps);
      L(cudaGetLastError());
      k_b_rinv<B, true, false><<<bt->n_rn, 128, 0, st>>>(pr, bt->d_rn, jp);
      L(cudaGetLastError());
    }
    nn_launch<B, NN_AX>(bt, L);
  }
  project();  // Y' = (I - Q Q^T) Y_j, twice
  orth_x(true);
  tn_launch<B, TN_QTA>(bt, bt->d_ctn, bt->ctn_off, L);
  k_b_indicator<B><<<(np + 127) / 128, 128, 0, st>>>(pr, np, jp, bt->d_part, bt->d_count);
  L(cudaGetLastError());
  if (graph)
    k_b_next<true><<<1, 1, 0, st>>>(bt->d_j, bt->d_count, bt->max_steps, h, nullptr);
  else
    k_b_next<false><<<1, 1, 0, st>>>(bt->d_j, bt->d_count, bt->max_steps, h, bt->d_more);
  L(cudaGetLastError());
  bt->launches_per_step = n;
  return first;
}

template <int B>
cudaError_t capture_step(lra_batch* bt, cudaGraph_t body, cudaGraphConditionalHandle h) {
  cudaError_t e = cudaStreamBeginCaptureToGraph(bt->st, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t ei = issue_step<B>(bt, true, h);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(bt->st, &g);
  return ei != cudaSuccess ? ei : ec;
}

cudaError_t issue_step_any(lra_batch* bt) {
  cudaGraphConditionalHandle h{};
  if (bt->b == 8) return issue_step<8>(bt, false, h);
  if (bt->b == 16) return issue_step<16>(bt, false, h);
  return issue_step<32>(bt, false, h);
}

cudaError_t build_graph(lra_batch* bt) {
  cudaError_t e = cudaGraphCreate(&bt->graph, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, bt->graph, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, bt->graph, nullptr, nullptr, 0, &cp);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (bt->b == 8)
    e = capture_step<8>(bt, body, h);
  else if (bt->b == 16)
    e = capture_step<16>(bt, body, h);
  else
    e = capture_step<32>(bt, body, h);
  if (e != cudaSuccess) return e;
  return cudaGraphInstantiate(&bt->exec, bt->graph, 0);
}

// Re-plans the tunable tile lists for tiling tl (the order and the pool stay),
// uploads them with the problems' records (which also resets the problems' state:
// lra_batch_run re-initialises it anyway) and rebuilds the step graph.
cudaError_t apply_tiling(lra_batch* bt, const BatchTiling& tl) {
  const BatchPlan plan = make_batch_plan(bt->ms, bt->ns, bt->b, bt->max_blocks, ZMAX, tl);
  std::vector<BProb> h = bt->h_init;
  for (int k = 0; k < bt->np; ++k) {
    const BatchProblemPlan& pp = plan.prob[k];
    h[k].g64_first = pp.g64_first;
    h[k].g64_count = pp.g64_count;
  }
  cudaError_t e = cudaStreamSynchronize(bt->st);  // nothing of an earlier run reads the lists
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bt->d_pr, h.data(), sizeof(BProb) * bt->np, cudaMemcpyHostToDevice, bt->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bt->d_ctn, plan.ctn.data(), sizeof(int2) * plan.ctn.size(), cudaMemcpyHostToDevice,
                        bt->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bt->d_qtn, plan.qtn.data(), sizeof(int2) * plan.qtn.size(), cudaMemcpyHostToDevice,
                        bt->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bt->d_rnn, plan.rnn.data(), sizeof(int2) * plan.rnn.size(), cudaMemcpyHostToDevice,
                        bt->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(bt->st);  // h is a local
  if (e != cudaSuccess) return e;
  for (int c = 0; c <= BATCH_CLASSES; ++c) {
    bt->ctn_off[c] = plan.ctn_off[c];
    bt->qtn_off[c] = plan.qtn_off[c];
    bt->rnn_off[c] = plan.rnn_off[c];
  }
  bt->tiling = tl;
  bt->h_pr = h;
  if (!bt->graph_mode) return cudaSuccess;
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  bt->exec = nullptr;
  bt->graph = nullptr;
  return build_graph(bt);
}

void batch_free(lra_batch* bt) {
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  void* ptrs[] = {bt->d_pr, bt->d_c32, bt->d_ctn, bt->d_rm, bt->d_rn, bt->d_qtn, bt->d_rnn, bt->d_part,
                  bt->d_j,  bt->d_count, bt->d_more, bt->d_pool};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (bt->own_stream && bt->st) cudaStreamDestroy(bt->st);
  delete bt;
}

}  // namespace
}  // namespace lra

extern "C" {

lra_status lra_batch_create(lra_batch** out, const lra_batch_item* items, int64_t count,
                            const lra_batch_params* prm, void* cuda_stream) {
  using namespace lra;
  if (!out || !items || !prm || count < 1 || count > (1 << 24)) return LRA_ERR_INVALID_ARG;
  *out = nullptr;
  const int B = prm->b;
  if ((B != 8 && B != 16 && B != 32) || prm->P < 0 || prm->P > 1 || prm->zeta < 1 ||
      prm->zeta > ZMAX || prm->max_blocks < 0 || (prm->flags & ~LRA_FLAG_NO_GRAPHS))
    return LRA_ERR_INVALID_ARG;
  for (int64_t i = 0; i < count; ++i) {
    const lra_batch_item& it = items[i];
    if (!it.A || it.m < 1 || it.n < 1 || it.lda < it.m || it.m > (1 << 30) || it.n > (1 << 30) ||
        B > std::min(it.m, it.n) || prm->zeta > it.n || !(it.eps > 0.0 && isfinite(it.eps)))
      return LRA_ERR_INVALID_ARG;
  }
  lra_batch* bt = new lra_batch();
  bt->np = (int)count;
  bt->b = B;
  bt->P = prm->P;
  bt->st = (cudaStream_t)cuda_stream;
  if (!bt->st) {
    if (cudaStreamCreate(&bt->st) != cudaSuccess) {
      delete bt;
      return LRA_ERR_CUDA;
    }
    bt->own_stream = true;
  }
  // order, caps, pool offsets and tile lists (batch_plan.h)
  std::vector<int64_t> ms(count), ns(count);
  for (int64_t i = 0; i < count; ++i) {
    ms[i] = items[i].m;
    ns[i] = items[i].n;
  }
  const BatchPlan plan = make_batch_plan(ms, ns, B, prm->max_blocks, ZMAX);
  // the tunable lists are largest with one column or row per thread
  const BatchTiling finest{{1, 1, 1}, {1, 1, 1}};
  const BatchPlan fine = make_batch_plan(ms, ns, B, prm->max_blocks, ZMAX, finest);
  static_assert(sizeof(BatchTile) == sizeof(int2), "tile lists are read as int2 on the device");
  const std::vector<BatchTile>& c32 = plan.c32;
  const std::vector<BatchTile>& rm = plan.rm;
  const std::vector<BatchTile>& rn = plan.rn;
  bt->order = plan.order;
  bt->ms = ms;
  bt->ns = ns;
  bt->max_blocks = prm->max_blocks;
  std::vector<BProb> h(count);
  for (int k = 0; k < (int)count; ++k) {
    const lra_batch_item& it = items[plan.ord[k]];
    const BatchProblemPlan& pp = plan.prob[k];
    BProb& p = h[k];
    memset(&p, 0, sizeof p);
    p.A = it.A;
    p.lda = it.lda;
    p.m = (int)it.m;
    p.n = (int)it.n;
    p.zeta = prm->zeta;
    p.cap = pp.cap;
    p.lmax = pp.lmax;
    p.eps2 = it.eps * it.eps;
    p.k0 = (uint32_t)(it.seed & 0xFFFFFFFFull);
    p.k1 = (uint32_t)(it.seed >> 32);
    p.c32_first = pp.c32_first;
    p.c32_count = pp.c32_count;
  }
  bt->max_steps = plan.max_steps;
  const int64_t off = plan.pool_bytes;
  bt->pool_bytes = off;
  bt->n_c32 = (int)c32.size();
  bt->n_rm = (int)rm.size();
  bt->n_rn = (int)rn.size();
  cudaError_t e = cudaMalloc((void**)&bt->d_pool, (size_t)std::max<int64_t>(off, 256));
  if (e == cudaSuccess) e = cudaMalloc((void**)&bt->d_pr, sizeof(BProb) * count);
  if (e == cudaSuccess) e = cudaMalloc((void**)&bt->d_c32, sizeof(int2) * c32.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&bt->d_rm, sizeof(int2) * rm.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&bt->d_rn, sizeof(int2) * rn.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&bt->d_qtn, sizeof(int2) * fine.qtn.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&bt->d_ctn, sizeof(int2) * fine.ctn.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&bt->d_rnn, sizeof(int2) * fine.rnn.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&bt->d_part, sizeof(double) * c32.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&bt->d_j, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&bt->d_count, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&bt->d_more, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_free(bt);
    return e == cudaErrorMemoryAllocation ? LRA_ERR_OOM : LRA_ERR_CUDA;
  }
  for (int k = 0; k < (int)count; ++k) {
    BProb& p = h[k];
    char* base = bt->d_pool;
    const int64_t* o = plan.prob[k].offs;
    p.Q = (float*)(base + o[0]);
    p.Bt = (float*)(base + o[1]);
    p.X = (float*)(base + o[2]);
    p.W = (float*)(base + o[3]);
    p.F = (float*)(base + o[5]);
    p.Rinv = (float*)(base + o[6]);
    p.omv = (float*)(base + o[7]);
    p.omr = (int*)(base + o[8]);
    p.rdiag = (double*)(base + o[9]);
    p.cnorm = (double*)(base + o[10]);
  }
  bt->h_init = h;
  e = cudaMemcpyAsync(bt->d_c32, c32.data(), sizeof(int2) * c32.size(), cudaMemcpyHostToDevice, bt->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bt->d_rm, rm.data(), sizeof(int2) * rm.size(), cudaMemcpyHostToDevice, bt->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bt->d_rn, rn.data(), sizeof(int2) * rn.size(), cudaMemcpyHostToDevice, bt->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->d_pool, 0, (size_t)off, bt->st);
  bt->graph_mode = (prm->flags & LRA_FLAG_NO_GRAPHS) == 0;
  // the tile lists and problem records of the default tiling, and the graph
  if (e == cudaSuccess) e = apply_tiling(bt, batch_default_tiling());
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_free(bt);
    return LRA_ERR_CUDA;
  }
  *out = bt;
  return LRA_OK;
}

lra_status lra_batch_run(lra_batch* bt) {
  using namespace lra;
  if (!bt) return LRA_ERR_INVALID_ARG;
  k_b_norm<<<bt->n_c32, 256, 0, bt->st>>>(bt->d_pr, bt->d_c32, bt->d_part);
  cudaError_t e = launched();
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->d_count, 0, sizeof(int), bt->st);
  if (e == cudaSuccess) {
    k_b_start<<<(bt->np + 127) / 128, 128, 0, bt->st>>>(bt->d_pr, bt->np, bt->d_part, bt->d_j);
    e = launched();
  }
  if (e == cudaSuccess && bt->graph_mode) e = cudaGraphLaunch(bt->exec, bt->st);
  // without the graph: one step at a time, the host reads whether to go on
  for (int j = 0; e == cudaSuccess && !bt->graph_mode && j < bt->max_steps; ++j) {
    e = issue_step_any(bt);
    int more = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&more, bt->d_more, sizeof(int), cudaMemcpyDeviceToHost, bt->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(bt->st);
    if (e == cudaSuccess) g_launches.fetch_add(bt->launches_per_step);
    if (!more) break;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bt->h_pr.data(), bt->d_pr, sizeof(BProb) * bt->np, cudaMemcpyDeviceToHost,
                        bt->st);
  int steps = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&steps, bt->d_j, sizeof(int), cudaMemcpyDeviceToHost, bt->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(bt->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LRA_ERR_CUDA;
  }
  bt->steps_last = steps;
  if (bt->graph_mode) g_launches.fetch_add((uint64_t)steps * bt->launches_per_step);
  return LRA_OK;
}

lra_status lra_batch_result(const lra_batch* bt, int64_t i, lra_batch_result_t* out) {
  if (!bt || !out || i < 0 || i >= bt->np) return LRA_ERR_INVALID_ARG;
  const lra::BProb& p = bt->h_pr[bt->order[i]];
  memset(out, 0, sizeof *out);
  out->status = p.status;
  out->rank = p.rank;
  out->E = p.E;
  out->normA2 = p.normA2;
  out->rel_err = p.normA2 > 0.0 ? sqrt(std::max(p.E, 0.0) / p.normA2) : 0.0;
  out->Q = p.Q;
  out->ldq = p.m;
  out->Bt = p.Bt;
  out->ldbt = p.n;
  return LRA_OK;
}

int64_t lra_batch_steps(const lra_batch* bt) { return bt ? bt->steps_last : -1; }

int64_t lra_batch_device_bytes(const lra_batch* bt) { return bt ? bt->pool_bytes : -1; }

lra_status lra_batch_set_tiling(lra_batch* bt, const lra_batch_tiling* t) {
  using namespace lra;
  if (!bt || !t) return LRA_ERR_INVALID_ARG;
  BatchTiling tl;
  for (int c = 0; c < BATCH_CLASSES; ++c) {
    tl.tn[c] = t->tn[c];
    tl.nn[c] = t->nn[c];
  }
  if (!batch_tiling_valid(tl)) return LRA_ERR_INVALID_ARG;
  if (apply_tiling(bt, tl) != cudaSuccess) {
    cudaGetLastError();
    return LRA_ERR_CUDA;
  }
  return LRA_OK;
}

lra_status lra_batch_get_tiling(const lra_batch* bt, lra_batch_tiling* t) {
  if (!bt || !t) return LRA_ERR_INVALID_ARG;
  for (int c = 0; c < lra::BATCH_CLASSES; ++c) {
    t->tn[c] = bt->tiling.tn[c];
    t->nn[c] = bt->tiling.nn[c];
  }
  return LRA_OK;
}

lra_status lra_batch_tune(lra_batch* bt, int32_t reps, lra_batch_tiling* best, double* best_ms,
                          double* base_ms) {
  using namespace lra;
  if (!bt || reps < 1) return LRA_ERR_INVALID_ARG;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return LRA_ERR_CUDA;
  }
  // ms per run of tiling tl (minimum over reps), or a negative value on an error
  auto time_of = [&](const BatchTiling& tl) -> double {
    if (apply_tiling(bt, tl) != cudaSuccess) return -1.0;
    double best_t = -1.0;
    for (int r = 0; r < reps; ++r) {
      if (cudaEventRecord(e0, bt->st) != cudaSuccess) return -1.0;
      if (lra_batch_run(bt) != LRA_OK) return -1.0;
      float ms = 0.f;
      if (cudaEventRecord(e1, bt->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        return -1.0;
      if (best_t < 0.0 || ms < best_t) best_t = ms;
    }
    return best_t;
  };
  // the classes the batch holds
  bool has_tn[BATCH_CLASSES] = {}, has_nn[BATCH_CLASSES] = {};
  for (int i = 0; i < bt->np; ++i) {
    has_tn[batch_tn_class(bt->ns[i])] = true;
    has_nn[batch_nn_class(bt->ms[i])] = true;
  }
  BatchTiling cur = bt->tiling;
  double cur_t = time_of(cur);
  const double base_t = cur_t;
  lra_status st = cur_t < 0.0 ? LRA_ERR_CUDA : LRA_OK;
  for (int knob = 0; st == LRA_OK && knob < 2 * BATCH_CLASSES; ++knob) {
    const int c = knob % BATCH_CLASSES;
    const bool is_tn = knob < BATCH_CLASSES;
    if (!(is_tn ? has_tn[c] : has_nn[c])) continue;
    for (int v : {1, 2, 4}) {
      BatchTiling cand = cur;
      int& slot = is_tn ? cand.tn[c] : cand.nn[c];
      if (slot == v) continue;
      slot = v;
      const double t = time_of(cand);
      if (t < 0.0) {
        st = LRA_ERR_CUDA;
        break;
      }
      if (t < cur_t) {
        cur = cand;
        cur_t = t;
      }
    }
  }
  if (st == LRA_OK && apply_tiling(bt, cur) != cudaSuccess) st = LRA_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LRA_OK) {
    cudaGetLastError();
    return st;
  }
  if (best)
    for (int c = 0; c < BATCH_CLASSES; ++c) {
      best->tn[c] = cur.tn[c];
      best->nn[c] = cur.nn[c];
    }
  if (best_ms) *best_ms = cur_t;
  if (base_ms) *base_ms = base_t;
  return LRA_OK;
}

void lra_batch_destroy(lra_batch* bt) {
  if (!bt) return;
  if (bt->st) cudaStreamSynchronize(bt->st);
  lra::batch_free(bt);
}

}  // extern "C"
