// FP64 skinny GEMM on the CUDA cores: C = alpha op(X) Y + beta C with N <= 64.
// Serves every dense contraction of the farPCA block (arxiv 2506.03859 Alg. 1
// steps A^T(A G_j), A G_j, A^T Y_j; the projections Q^T Y, Q F; the deflation
// B^T (B Omega); the b x b Gram matrices).  On GB300 the FP64 pipe (about
// 1.2 TFLOP/s measured) bounds it, not HBM: every element of X is used N times.
//
// Tiling: a CTA owns 64 rows p of the output and all N <= 64 columns, walks its
// K range in steps of 16 staged through shared memory, and each of its 256
// threads accumulates a 4 x 4 block (rows tp + 16i, columns tc + 16j).  When
// the output has too few row tiles to fill the GPU the K range is split across
// CTAs; partial tiles go to a workspace and a second kernel sums them in a
// fixed order (deterministic results).
#include "internal.cuh"

namespace lra {

namespace {
constexpr int TP = 64, TN = 64, TK = 16, NT = 256;
constexpr int64_t WS_TILES = 640;  // split tiles the workspace holds
constexpr int TARGET_CTAS = 2 * 152;
}  // namespace

int64_t dgemm_ws_elems() { return WS_TILES * TP * TN; }

template <bool TRANS>
__global__ void __launch_bounds__(NT)
    k_dgemm(int64_t P, int N, int64_t K, int64_t kchunk, double alpha,
            const double* __restrict__ X, int64_t ldx, const double* __restrict__ Y, int64_t ldy,
            double beta, double* __restrict__ C, int64_t csp, int64_t csc,
            double* __restrict__ ws, int64_t ppad) {
  __shared__ double Xs[TK][TP + 1];
  __shared__ double Ys[TK][TN + 1];
  const int tid = threadIdx.x;
  const int64_t p0 = (int64_t)blockIdx.x * TP;
  const int64_t kb = (int64_t)blockIdx.y * kchunk;
  const int64_t ke = (kb + kchunk < K) ? kb + kchunk : K;
  const int tp = tid & 15, tc = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = kb; k0 < ke; k0 += TK) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (TRANS) {
        const int kk = tid & 15, pp = (tid >> 4) + 16 * s;
        const int64_t k = k0 + kk, p = p0 + pp;
        Xs[kk][pp] = (k < ke && p < P) ? __ldg(X + k + p * ldx) : 0.0;
      } else {
        const int pp = tid & 63, kk = (tid >> 6) + 4 * s;
        const int64_t k = k0 + kk, p = p0 + pp;
        Xs[kk][pp] = (k < ke && p < P) ? __ldg(X + p + k * ldx) : 0.0;
      }
      const int kk = tid & 15, cc = (tid >> 4) + 16 * s;
      const int64_t k = k0 + kk;
      Ys[kk][cc] = (k < ke && cc < N) ? __ldg(Y + k + (int64_t)cc * ldy) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double xr[4], yr[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xr[i] = Xs[kk][tp + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) yr[j] = Ys[kk][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(xr[i], yr[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t p = p0 + tp + 16 * i;
    if (p >= P) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = tc + 16 * j;
      if (c >= N) continue;
      if (ws) {
        ws[((int64_t)blockIdx.y * TN + c) * ppad + p] = acc[i][j];
      } else {
        double* dst = C + p * csp + (int64_t)c * csc;
        *dst = (beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*dst);
      }
    }
  }
}

__global__ void k_splitk_reduce(int64_t P, int N, int splits, int64_t ppad,
                                const double* __restrict__ ws, double alpha, double beta,
                                double* __restrict__ C, int64_t csp, int64_t csc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P * N) return;
  const int64_t p = idx % P;
  const int c = (int)(idx / P);
  double s = 0.0;
  for (int q = 0; q < splits; ++q) s += ws[((int64_t)q * TN + c) * ppad + p];
  double* dst = C + p * csp + (int64_t)c * csc;
  *dst = (beta == 0.0) ? alpha * s : alpha * s + beta * (*dst);
}

cudaError_t dgemm(bool trans, int64_t P, int64_t N, int64_t K, double alpha, const double* X,
                  int64_t ldx, const double* Y, int64_t ldy, double beta, GemmOut out, double* ws,
                  int64_t ws_elems, cudaStream_t st) {
  if (P <= 0 || N <= 0) return cudaSuccess;
  if (N > TN) return cudaErrorInvalidValue;
  const int64_t ptiles = (P + TP - 1) / TP;
  int64_t splits = 1;
  if (K > 512 && ptiles < TARGET_CTAS) {
    splits = (TARGET_CTAS + ptiles - 1) / ptiles;
    const int64_t by_k = (K + 255) / 256;
    if (splits > by_k) splits = by_k;
    const int64_t by_ws = ws_elems / (ptiles * TP * TN);
    if (splits > by_ws) splits = by_ws;
    if (splits < 1) splits = 1;
  }
  int64_t kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + TK - 1) / TK * TK;
  if (kchunk < TK) kchunk = TK;
  splits = (K + kchunk - 1) / kchunk;
  if (splits < 1) splits = 1;
  const int64_t ppad = ptiles * TP;
  dim3 grid((unsigned)ptiles, (unsigned)splits);
  double* wsp = (splits > 1) ? ws : nullptr;
  if (trans)
    k_dgemm<true><<<grid, NT, 0, st>>>(P, (int)N, K, kchunk, alpha, X, ldx, Y, ldy, beta, out.C,
                                       out.csp, out.csc, wsp, ppad);
  else
    k_dgemm<false><<<grid, NT, 0, st>>>(P, (int)N, K, kchunk, alpha, X, ldx, Y, ldy, beta, out.C,
                                        out.csp, out.csc, wsp, ppad);
  cudaError_t e = launched();
  if (e != cudaSuccess || splits == 1) return e;
  const int64_t total = P * N;
  k_splitk_reduce<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, (int)N, (int)splits, ppad, ws,
                                                                  alpha, beta, out.C, out.csp,
                                                                  out.csc);
  return launched();
}

}  // namespace lra
