// FP64-accurate skinny GEMM on the tcgen05 tensor cores: C = alpha op(X) Y + beta C
// with X, Y, C in FP64 and N <= 64.  These are the full passes over A of the
// farPCA block (arxiv 2506.03859 Alg. 1 steps A^T(A G_j), A G_j, A^T Y_j) and the
// smaller products of the projection and orthonormalisation steps.
//
// GB300's FP64 pipe delivers about 1.2 TFLOP/s, while such a pass streams A once
// from HBM: run as FP64 FMAs it is ~60x slower than the memory bound.  Instead
// every operand is cut, error-free, into small integer digits that the 16-bit
// tensor-core formats hold exactly (the splitting idea of Ozaki, Ogita, Oishi,
// Rump, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms 2012):
//
//   Scaling.  Row p of op(X) has largest biased exponent ex_p, column c of Y
//   ey_c.  x is turned into the signed integer N = trunc(x 2^(1077 - ex_p)),
//   |N| < 2^55, and written in base 256 with seven digits d_0..d_6 (d_0 the most
//   significant): N = sum_s d_s 256^(6-s), d_0 in [-128, 128], d_1..6 in
//   [-128, 127], stored as f16 (exact).  Y is cut the same way into e_0..e_6.
//
//   Products.  x y = 2^(ex + ey - 2058) sum_{s,t} d_s e_t 256^(-(s+t)).  The 28
//   pairs of weight w = s + t <= 6 are kept (the dropped ones are below 2^-53 of
//   max|x| max|y|).  For each weight w the tensor core sums G_w = sum_{s+t=w}
//   sum_k d_s e_t in an FP32 accumulator in TMEM (columns 64 w .. 64 w + 63).
//
//   Exact part.  For w <= 3 and a window of at most 64 values of K, |G_w| <=
//   4 * 64 * 128^2 = 2^22, so the FP32 accumulator holds it exactly.  The
//   accumulator starts each window at 1.5 * 2^23; its bit pattern minus that of
//   1.5 * 2^23 is then G_w as an integer, and the four are folded into one int64
//   per output, T += G_0 2^24 + G_1 2^16 + G_2 2^8 + G_3, held by the flush
//   warps (half in registers, half in spare TMEM columns; exact while K <= 2^24).
//
//   Rest.  G_4, G_5, G_6 (at most 2^-32 of the leading term) run in FP32 over
//   the whole range of K of the tile.  The result is
//   (T 2^-24 + G_4 2^-32 + G_5 2^-40 + G_6 2^-48) 2^(ex + ey - 2058), written in
//   FP64; against exact dot products its error is that of an FP64 GEMM.
//
// Tensor-core schedule.  Digit planes of Y are stored one after another in shared
// memory, so one MMA with X plane s and Y planes t..t+c-1 (N = 64 c <= 256)
// produces the weights s+t .. s+t+c-1 into adjacent TMEM column ranges: the 28
// pairs take 11 MMAs per 16 values of K (4 for w <= 3, 7 for w >= 4), one stage.
//
// Work split: one CTA per SM walks a contiguous range of (row tile, 16-deep
// stage) units ("stream-K"); tiles whose stages span two or more CTAs are
// written as partial sums and combined by a fixup kernel in a fixed order.
// Inside a CTA the work is pipelined by warp role: eight producer warps load a
// 128 x 16 block of op(X) one stage ahead into registers, cut it into the seven
// digit planes of a shared-memory stage (four stages, K-major core-matrix layout),
// while a bulk copy brings the pre-cut 64 x 16 block of Y; one thread issues
// the MMAs; four warps read the exact sums from TMEM at the end of each 64-deep
// window, re-arm them, and write the tile.  The MMAs of weight >= 4 of a window
// are issued before the wait for that re-arming, so the flush overlaps them.
// mbarriers hand stages and accumulators between the roles; every wait is bounded.
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>

#include "chol.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace lra {

namespace {
constexpr int S = 7;                     // digits per operand
constexpr int TM = 128;                  // rows of op(X) per tile
constexpr int KS = 16;                   // K per pipeline stage (one MMA k-step)
constexpr int NN = 64;                   // output columns (N padded)
constexpr int NFLUSH = 128;              // flush threads (warps 0..3)
constexpr int NPROD = 256;               // producer threads (warps 4..11)
constexpr int MMA_WARP = 12;
constexpr int NT = NFLUSH + NPROD + 32;
constexpr int A_PLANE = TM * KS * 2;     // bytes of one digit plane of the op(X) block
constexpr int Y_PLANE = NN * KS * 2;     // bytes of one digit plane of the Y block
constexpr int Y_STAGE = S * Y_PLANE;     // the Y part of a stage (one bulk copy)
constexpr int STAGE = S * A_PLANE + Y_STAGE;
constexpr int NSTAGE = 4;
constexpr int SMEM_DYN = NSTAGE * STAGE + 1024;
constexpr uint32_t LBO = 128, SBO = 256;  // core-matrix strides (K, rows)
constexpr uint32_t TMEM_COLS = 512;       // weights 0..6: columns 0..447
constexpr uint32_t COL_ACC_LO = 448, COL_ACC_HI = 480;  // int64 sums of output columns 32..63
constexpr uint32_t ACC_SET1 = 256;  // the reduced form's second set of exact sums (weights 0..3)
constexpr uint32_t MAGIC = 0x4B400000u;   // bits of 1.5 * 2^23
constexpr long WAIT_TRIES = 1L << 22;
constexpr int EXP_OFFSET = 2058;          // 2 * 1077 - 96: see the scaling above
constexpr int64_t MAX_K = int64_t(1) << 24;
}  // namespace

int64_t oz_img_bytes(int64_t K) { return (K + KS - 1) / KS * Y_STAGE; }
int64_t oz_part_elems(int ctas) { return (int64_t)ctas * 2 * TM * NN; }
int64_t oz_max_k() { return MAX_K; }

// Offset of element (row, k), k < 16, in the K-major core-matrix layout of a
// stage plane: core (row/8, k/8) at ((row/8)*2 + k/8)*128, row-major inside.
__host__ __device__ __forceinline__ uint32_t core_offset(uint32_t row, uint32_t k) {
  return (((row >> 3) << 1) + (k >> 3)) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

// N + BIAS as two 32-bit words, N = trunc(x 2^(1077 - emax)) (emax >= the
// biased exponent of x; zero and subnormal x give 0) and BIAS = 128 in each of
// the seven low bytes.  N + BIAS >= 0; its six low bytes u_1..u_6 and its bits
// 48.. (u_0 <= 256) give the digits d_s = u_s - 128 of N.  Branch-free: the
// significand M (53 bits) is shifted to M << 10 and right by min(k, 63), which
// clears it for every k >= 63.
__device__ __forceinline__ void biased_fixed(double x, int emax, uint32_t& nh, uint32_t& nl) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  const uint32_t h = (uint32_t)(bits >> 32);
  const int E = (int)((h >> 20) & 0x7FFu);
  const uint64_t M = (bits & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int k = min(E != 0 ? emax - E + 8 : 63, 63);
  const uint64_t a = (M << 10) >> k;                     // |N|
  const uint64_t sgn = (uint64_t)((int64_t)(int)h >> 63);  // 0, or all ones for negative x
  const uint64_t v = (a ^ sgn) + (0x0080808080808080ull + (sgn & 1u));
  nh = (uint32_t)(v >> 32);
  nl = (uint32_t)v;
}

// Digit SL (0 = most significant) of two values a, b as a packed f16 pair (a in
// the low half): the digit bytes (u + 1024 as f16 bits, i.e. 0x64uu) are built
// by a byte permute and a mask, and one packed f16 subtract removes 1024 + 128;
// every step is exact.
template <int SL>
__device__ __forceinline__ uint32_t digit_pair(uint32_t ha, uint32_t la, uint32_t hb, uint32_t lb) {
  uint32_t w;
  if (SL == 0) {
    w = __byte_perm(ha, hb, 0x7632u) + 0x64006400u;  // 16-bit top parts (<= 256) + 1024
  } else {
    constexpr uint32_t byte = (SL <= 2) ? (2 - SL) : (6 - SL);
    const uint32_t xa = (SL <= 2) ? ha : la, xb = (SL <= 2) ? hb : lb;
    w = (__byte_perm(xa, xb, byte | (byte << 4) | ((byte + 4) << 8) | ((byte + 4) << 12)) &
         0x00FF00FFu) | 0x64006400u;
  }
  const __half2 r = __hsub2(*reinterpret_cast<const __half2*>(&w), __half2(__half(1152.0f), __half(1152.0f)));
  return *reinterpret_cast<const uint32_t*>(&r);
}

// Eight consecutive K values of one row (or column) -> one 16-byte chunk in each
// of the seven digit planes at dst, dst + plane, ...
__device__ __forceinline__ void cut8(const double* v, int emax, uint8_t* dst, int plane) {
  uint32_t h[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) biased_fixed(v[i], emax, h[i], l[i]);
#define LRA_CUT(SL)                                                   \
  {                                                                   \
    uint4 q;                                                          \
    q.x = digit_pair<SL>(h[0], l[0], h[1], l[1]);                     \
    q.y = digit_pair<SL>(h[2], l[2], h[3], l[3]);                     \
    q.z = digit_pair<SL>(h[4], l[4], h[5], l[5]);                     \
    q.w = digit_pair<SL>(h[6], l[6], h[7], l[7]);                     \
    *reinterpret_cast<uint4*>(dst + (SL) * plane) = q;                \
  }
  LRA_CUT(0) LRA_CUT(1) LRA_CUT(2) LRA_CUT(3) LRA_CUT(4) LRA_CUT(5) LRA_CUT(6)
#undef LRA_CUT
}

// ---------------------------------------------------------------- prep kernels

// out[c] = largest biased exponent of X[:, c] (out pre-zeroed): CTA (c, y) scans
// rows [y rchunk, (y + 1) rchunk) of column c.
__global__ void __launch_bounds__(256) k_oz_colmaxexp(const double* __restrict__ X, int64_t ld,
                                                      int64_t rows, int64_t rchunk,
                                                      int* __restrict__ out,
                                                      const int* __restrict__ skip) {
  if (skip && __ldcg(skip)) return;
  __shared__ int red[8];
  const int64_t c = blockIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * rchunk;
  const int64_t r1 = (r0 + rchunk < rows) ? r0 + rchunk : rows;
  int e = 0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += 256) {
    const uint64_t b = (uint64_t)__double_as_longlong(__ldg(X + i + c * ld));
    e = max(e, (int)((b >> 52) & 0x7FFu));
  }
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_down_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int q = 0; q < 8; ++q) t = max(t, red[q]);
    if (gridDim.y == 1)
      out[c] = t;  // the only chunk: no zeroing, no atomics
    else
      atomicMax(out + c, t);
  }
}

// Column exponents of X (rows x cols): zero out, then the split scan.  skip: as
// for OzArgs (only with rows <= 4096, where nothing is zeroed).
cudaError_t colmaxexp(const double* X, int64_t ld, int64_t rows, int64_t cols, int* out,
                      cudaStream_t st, const int* skip = nullptr) {
  const int64_t rchunk = 4096;
  if (skip && rows > rchunk) return cudaErrorInvalidValue;
  if (rows > rchunk) {
    cudaError_t e = cudaMemsetAsync(out, 0, cols * sizeof(int), st);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)cols, (unsigned)((rows + rchunk - 1) / rchunk));
  k_oz_colmaxexp<<<grid, 256, 0, st>>>(X, ld, rows, rchunk, out, skip);
  return launched();
}

// out[r] = max over the columns of X[r, :] of the biased exponent (out pre-zeroed).
__global__ void __launch_bounds__(256) k_oz_rowmaxexp(const double* __restrict__ X, int64_t ld,
                                                      int64_t rows, int64_t cols, int64_t cchunk,
                                                      int* __restrict__ out, bool direct,
                                                      const int* __restrict__ skip) {
  if (skip && __ldcg(skip)) return;
  const int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (r >= rows) return;
  const int64_t c0 = (int64_t)blockIdx.y * cchunk;
  const int64_t c1 = (c0 + cchunk < cols) ? c0 + cchunk : cols;
  int e = 0;
  for (int64_t c = c0; c < c1; ++c) {
    const uint64_t b = (uint64_t)__double_as_longlong(__ldg(X + r + c * ld));
    e = max(e, (int)((b >> 52) & 0x7FFu));
  }
  if (direct)
    out[r] = e;  // one column chunk and nothing to accumulate: plain store
  else
    atomicMax(out + r, e);
}

// Pre-cut Y: stage u of the image holds the seven 64 x 16 (N x K) digit planes
// of K values 16u .. 16u + 15 in the core-matrix layout.  One thread per
// (stage, column c, 8-wide k chunk j).
__global__ void __launch_bounds__(256) k_oz_ycut(const double* __restrict__ Y, int64_t ldy,
                                                 int64_t K, int N, const int* __restrict__ yE,
                                                 uint8_t* __restrict__ img, int64_t kst,
                                                 const int* __restrict__ skip) {
  if (skip && __ldcg(skip)) return;
  const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (idx >= kst * NN * 2) return;
  const int j = (int)(idx & 1);
  const int c = (int)((idx >> 1) & (NN - 1));
  const int64_t u = idx >> 7;
  const int emax = c < N ? yE[c] : 0;
  double v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t k = u * KS + 8 * j + i;
    v[i] = (c < N && k < K) ? __ldg(Y + k + (int64_t)c * ldy) : 0.0;
  }
  cut8(v, emax, img + u * Y_STAGE + core_offset((uint32_t)c, (uint32_t)(8 * j)), Y_PLANE);
}

// ---------------------------------------------------------------- main kernel

struct OzArgs {
  int64_t P, K, N;
  const double* X;
  const float* X32;    // k_oz_xcut<TRANS, float>: X as float (converted exactly on load)
  int64_t ldx;
  const int* xE;       // biased max exponent of each row of op(X)
  const int* yE;       // biased max exponent of each column of Y
  const uint8_t* img;  // pre-cut Y
  double alpha, beta;
  double* C;
  int64_t csp, csc;
  double* part;        // [cta][2][NN][TM] partial tiles
  int64_t tiles, kst;  // row tiles; 16-deep stages per tile
  int* flags;
  bool vec;            // 16-byte loads allowed (trans layout)
  bool whole_tiles;    // ranges hold whole tiles: no tile is split, no fixup
  const int* skip;     // NULL, or the launch does nothing while *skip != 0
};

// The range [u0, u1) of CTA cta of G: an even share of all units ("stream-K"),
// or, with whole_tiles, an even share of whole tiles.
__device__ __forceinline__ void cta_range(const OzArgs& a, int64_t cta, int64_t G, int64_t& u0,
                                          int64_t& u1) {
  if (a.whole_tiles) {
    u0 = (cta * a.tiles / G) * a.kst;
    u1 = ((cta + 1) * a.tiles / G) * a.kst;
  } else {
    const int64_t T = a.tiles * a.kst;
    u0 = cta * T / G;
    u1 = (cta + 1) * T / G;
  }
}

// The CTA's stages: a contiguous range [u0, u1) of (tile, stage) units,
// tile-major, walked with a (tile, stage-in-tile) cursor.  A segment is the part
// of the range inside one tile; a window is up to four consecutive stages (64
// values of K) of a segment, aligned to stage indices divisible by four.
struct Cursor {
  int64_t tile;   // row tile of the current unit
  int ks;         // its stage within the tile
  int64_t i;      // its index within the CTA's range
  int64_t n;      // units in the range
  int kst;        // stages per tile
  __device__ __forceinline__ void next() {
    ++i;
    if (++ks == kst) {
      ks = 0;
      ++tile;
    }
  }
  __device__ __forceinline__ bool seg_first() const { return i == 0 || ks == 0; }
  __device__ __forceinline__ bool seg_last() const { return i + 1 == n || ks + 1 == kst; }
  __device__ __forceinline__ bool win_first() const { return seg_first() || (ks & 3) == 0; }
  __device__ __forceinline__ bool win_last() const { return seg_last() || (ks & 3) == 3; }
};

// A producer thread's share of one stage: 8 values of op(X).  TRANS == false:
// op(X)[p, k] = X[p + k*ldx], the thread takes row 32 (pw % 4) + lane and 8
// consecutive k (coalesced across the warp).  TRANS == true: op(X)[p, k] =
// X[k + p*ldx]; each warp instruction covers one 8 x 8 core matrix, lane ->
// (row r8 = lane % 8, k pair lane / 8): values 2i, 2i+1 belong to row
// 8 (pw / 2 + 4 i) + r8 and k 8 (pw % 2) + 2 (lane / 8) + {0, 1}.
constexpr int VPT = TM * KS / NPROD;  // values per producer thread per stage

template <typename T>
__device__ __forceinline__ const T* xsrc(const OzArgs& a);
template <>
__device__ __forceinline__ const double* xsrc<double>(const OzArgs& a) { return a.X; }
template <>
__device__ __forceinline__ const float* xsrc<float>(const OzArgs& a) { return a.X32; }

// T: element type of X in memory (float is converted exactly to double).
template <bool TRANS, typename T = double>
__device__ __forceinline__ void fetch(const OzArgs& a, int64_t tile, int ks, int pw, int lane,
                                      double (&v)[VPT]) {
  const T* X = xsrc<T>(a);
  if (!TRANS) {
    const int64_t p = tile * TM + 32 * (pw & 3) + lane, kb = (int64_t)ks * KS + 8 * (pw >> 2);
    const T* src = X + p + kb * a.ldx;
    if (p < a.P && kb + 8 <= a.K) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        v[i] = (double)__ldg(src);
        src += a.ldx;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        v[i] = (p < a.P && kb + i < a.K) ? (double)__ldg(src + i * a.ldx) : 0.0;
    }
  } else {
    const int r8 = lane & 7, q = lane >> 3;
    const int64_t p0 = tile * TM + (pw >> 1) * 8 + r8, k = (int64_t)ks * KS + (pw & 1) * 8 + 2 * q;
    const T* src = X + k + p0 * a.ldx;
    if (a.vec && tile * TM + TM <= a.P && k + 2 <= a.K) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if constexpr (sizeof(T) == 8) {
          const double2 t = __ldg(reinterpret_cast<const double2*>(src));
          v[2 * i] = t.x;
          v[2 * i + 1] = t.y;
        } else {
          const float2 t = __ldg(reinterpret_cast<const float2*>(src));
          v[2 * i] = (double)t.x;
          v[2 * i + 1] = (double)t.y;
        }
        src += 32 * a.ldx;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const bool in = p0 + 32 * i < a.P;
        const T* s2 = src + 32 * i * a.ldx;
        v[2 * i] = (in && k < a.K) ? (double)__ldg(s2) : 0.0;
        v[2 * i + 1] = (in && k + 1 < a.K) ? (double)__ldg(s2 + 1) : 0.0;
      }
    }
  }
}

// Cut the thread's 8 values into the stage; sE = row exponents of the tile.
template <bool TRANS>
__device__ __forceinline__ void cut_stage(const double (&v)[VPT], const int* sE, uint8_t* sA, int pw,
                                          int lane) {
  if (!TRANS) {
    const uint32_t row = 32 * (pw & 3) + lane, kb = 8 * (pw >> 2);
    cut8(v, sE[row], sA + core_offset(row, kb), A_PLANE);
  } else {
    const int r8 = lane & 7, q = lane >> 3;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int core = pw + 8 * i;  // row group core / 2 = pw / 2 + 4 i, k group pw % 2
      const int e = sE[(core >> 1) * 8 + r8];
      uint8_t* dst = sA + core * 128 + r8 * 16 + q * 4;
      uint32_t h0, l0, h1, l1;
      biased_fixed(v[2 * i], e, h0, l0);
      biased_fixed(v[2 * i + 1], e, h1, l1);
#define LRA_CUT2(SL) \
  *reinterpret_cast<uint32_t*>(dst + (SL) * A_PLANE) = digit_pair<SL>(h0, l0, h1, l1);
      LRA_CUT2(0) LRA_CUT2(1) LRA_CUT2(2) LRA_CUT2(3) LRA_CUT2(4) LRA_CUT2(5) LRA_CUT2(6)
#undef LRA_CUT2
    }
  }
}

// One MMA of X digit plane s against Y planes t0 .. t0+c-1 (N = 64 c) into the
// weight columns 64 (s + t0) .. 64 (s + t0 + c) - 1, over the stage's 16 values of K.
__device__ __forceinline__ void mma_group(uint32_t tmem, uint32_t a0, uint32_t y0, int s, int t0,
                                          int c, uint32_t accumulate) {
  const uint32_t idesc = tc::idesc_f16_f32(TM, 64u * (uint32_t)c);
  tc::mma_f16(tmem + 64u * (uint32_t)(s + t0), tc::desc_k_none(a0 + (uint32_t)s * A_PLANE, LBO, SBO),
              tc::desc_k_none(y0 + (uint32_t)t0 * Y_PLANE, LBO, SBO), idesc, accumulate);
}

// Barriers, TMEM address and small tables a CTA's roles share.
struct OzShared {
  // accfull / accempty [set]: the exact sums of a window in accumulator set 0
  // (columns 0..255), or, in the reduced form, alternately in sets 0 and 1
  // (columns 256..511, free there), so that one window's MMAs run while the flush
  // folds the previous window's sums
  uint64_t full[NSTAGE], empty[NSTAGE], accfull[2], accempty[2];
  uint32_t tmem;
  int abort;
  int yE[NN];
};

// Set-up common to both kernels: TMEM (warp 0), barriers (thread 0), Y exponents.
// full_count: arrivals that complete a stage.
__device__ __forceinline__ void oz_setup(OzShared& sh, const OzArgs& a, int full_count,
                                         int flush_threads) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc::tmem_alloc(&sh.tmem, TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      tc::mbar_init(&sh.full[s], full_count);
      tc::mbar_init(&sh.empty[s], 1);
    }
    for (int a2 = 0; a2 < 2; ++a2) {
      tc::mbar_init(&sh.accfull[a2], 1);
      tc::mbar_init(&sh.accempty[a2], flush_threads);
    }
    sh.abort = 0;
  }
  if (tid < NN) sh.yE[tid] = tid < a.N ? a.yE[tid] : 0;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

__device__ __forceinline__ void oz_teardown(OzShared& sh, const OzArgs& a) {
  tc::fence_before_sync();
  __syncthreads();
  if (sh.abort && threadIdx.x == 0) atomicOr(a.flags, FLAG_TIMEOUT);
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(sh.tmem, TMEM_COLS);
}

// The MMA issuer (one thread).  Per stage: the weight >= 4 MMAs (FP32 over the
// segment; the first MMA of a segment starts them), then the exact weights 0..3,
// which at a window start must wait until the flush has read and re-armed them.
// To hide that wait the first two stages of a window are issued together: both
// stages' weight >= 4 MMAs, the wait, then both stages' exact MMAs.  A new
// segment first waits for the flush to finish the previous one (its FP32 sums).
// HIGH = false: the reduced form (digits 0..3 of both operands only), exact MMAs alone.
// YD1: Y has a single nonzero digit plane (plane 0, e.g. a +-1/2 test matrix), so the
// only nonzero pairs are (s, 0): one MMA of N = 64 per X plane, weight s.
template <bool HIGH, bool YD1 = false>
__device__ __forceinline__ void oz_mma_role(OzShared& sh, const Cursor& start, uint8_t* sm) {
  volatile int& s_abort = sh.abort;
  const uint32_t tmem = sh.tmem;
  uint32_t ph_full = 0, ph_ae = 0;  // ph_full bit s: the phase of full[s]
  auto wait_full = [&](int st) -> bool {
    if (!tc::mbar_wait(&sh.full[st], (ph_full >> st) & 1u, WAIT_TRIES)) return false;
    ph_full ^= 1u << st;
    tc::fence_after_sync();
    return true;
  };
  auto wait_accempty = [&]() -> bool {
    if (!tc::mbar_wait(&sh.accempty[0], ph_ae, WAIT_TRIES)) return false;
    ph_ae ^= 1u;
    tc::fence_after_sync();
    return true;
  };
  auto high = [&](int st, bool fresh) {
    if (!HIGH) return;
    const uint32_t a0 = tc::smem_addr(sm + st * STAGE), y0 = a0 + S * A_PLANE;
    if (YD1) {
      mma_group(tmem, a0, y0, 4, 0, 1, fresh ? 0u : 1u);
      mma_group(tmem, a0, y0, 5, 0, 1, fresh ? 0u : 1u);
      mma_group(tmem, a0, y0, 6, 0, 1, fresh ? 0u : 1u);
      return;
    }
    mma_group(tmem, a0, y0, 0, 4, 3, fresh ? 0u : 1u);
    mma_group(tmem, a0, y0, 1, 3, 3, 1u);
    mma_group(tmem, a0, y0, 2, 2, 3, 1u);
    mma_group(tmem, a0, y0, 3, 1, 3, 1u);
    mma_group(tmem, a0, y0, 4, 0, 3, 1u);
    mma_group(tmem, a0, y0, 5, 0, 2, 1u);
    mma_group(tmem, a0, y0, 6, 0, 1, 1u);
  };
  auto exact = [&](int st, uint32_t acc_col = 0u) {
    const uint32_t a0 = tc::smem_addr(sm + st * STAGE), y0 = a0 + S * A_PLANE;
    const uint32_t t0 = tmem + acc_col;
    if (YD1) {
      mma_group(t0, a0, y0, 0, 0, 1, 1u);
      mma_group(t0, a0, y0, 1, 0, 1, 1u);
      mma_group(t0, a0, y0, 2, 0, 1, 1u);
      mma_group(t0, a0, y0, 3, 0, 1, 1u);
      tc::mma_commit(&sh.empty[st]);
      return;
    }
    mma_group(t0, a0, y0, 0, 0, 4, 1u);
    mma_group(t0, a0, y0, 1, 0, 3, 1u);
    mma_group(t0, a0, y0, 2, 0, 2, 1u);
    mma_group(t0, a0, y0, 3, 0, 1, 1u);
    tc::mma_commit(&sh.empty[st]);
  };
  Cursor c = start;
  if (!HIGH) {
    // the reduced form: window w's exact sums in set w % 2; its MMAs wait only for
    // the fold of window w - 2 (the same set), not of window w - 1
    int set = 0;
    uint32_t ph_e2 = 0;  // bit s: the phase of accempty[s]
    while (c.i < c.n) {
      const int st = (int)(c.i % NSTAGE);
      if (!wait_full(st)) break;
      if (c.win_first()) {
        if (!tc::mbar_wait(&sh.accempty[set], (ph_e2 >> set) & 1u, WAIT_TRIES)) break;
        ph_e2 ^= 1u << set;
        tc::fence_after_sync();
      }
      exact(st, set ? ACC_SET1 : 0u);
      if (c.win_last()) {
        tc::mma_commit(&sh.accfull[set]);
        set ^= 1;
      }
      c.next();
    }
    if (c.i < c.n) s_abort = 1;
    return;
  }
  while (c.i < c.n) {
    const int st = (int)(c.i % NSTAGE);
    if (!wait_full(st)) break;
    const bool sf = c.seg_first();
    if (sf && !wait_accempty()) break;
    high(st, sf);
    if (c.win_first() && !sf) {
      if (!c.win_last()) {  // pair with the window's second stage
        Cursor d = c;
        d.next();
        const int st2 = (int)(d.i % NSTAGE);
        if (!wait_full(st2)) break;
        high(st2, false);
        if (!wait_accempty()) break;
        exact(st);
        exact(st2);
        if (d.win_last()) tc::mma_commit(&sh.accfull[0]);
        c = d;
        c.next();
        continue;
      }
      if (!wait_accempty()) break;
    }
    exact(st);
    if (c.win_last()) tc::mma_commit(&sh.accfull[0]);
    c.next();
  }
  if (c.i < c.n) s_abort = 1;
}

// v 2^e: the exponent field moves when the result stays normal, else ldexp.
__device__ __forceinline__ double scale2(double v, int e) {
  const int64_t bits = __double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex != 0 && ex + e > 0 && ex + e < 2047) return __longlong_as_double(bits + ((int64_t)e << 52));
  return ldexp(v, e);
}

// The flush (warps 0..3): at every window end fold the exact sums into the int64
// totals and re-arm them; at a segment end also read weights 4..6 and write the
// tile (to C when the segment is the whole tile, else to the CTA's partial slot).
// The flush (warps 0 .. NFW-1): at every window end fold the exact sums into the
// int64 totals and re-arm them; at a segment end also read weights 4..6 and write
// the tile (to C when the segment is the whole tile, else to the CTA's partial
// slot).  Warp w owns TMEM lanes / tile rows 32 (w % 4) .. + 31 (one row per
// thread).  NFW = 4: each warp takes all 64 output columns, the int64 sums of
// columns 0..31 in registers and of 32..63 in TMEM (COL_ACC_LO / COL_ACC_HI);
// NFW = 8: warps w and w + 4 split the columns, 32 each, all sums in registers.
// PIPE: overlap the TMEM loads of the next 4-column chunk with the current one
// (needs ~48 more registers; the on-the-fly kernel, capped at 128, goes without).
// HIGH = false: the reduced form, no weights 4..6.
template <bool PIPE, bool HIGH, int NFW>
__device__ __forceinline__ void oz_flush_role(OzShared& sh, const OzArgs& a, const Cursor& start,
                                              int64_t cta) {
  constexpr int NCOL = NFW == 8 ? 32 : 64;  // output columns per thread
  constexpr int NJ = NCOL / 4;              // 4-column chunks
  volatile int& s_abort = sh.abort;
  const int* syE = sh.yE;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, col0 = NFW == 8 ? NCOL * (warp >> 2) : 0;
  const int64_t first_tile = start.tile;
  static_assert(HIGH || NFW == 8, "the reduced form keeps its totals in registers");
  const uint32_t tb = sh.tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)col0;
#pragma unroll
  for (int w = 0; w < 4; ++w)
#pragma unroll
    for (int j = 0; j < NCOL / 8; ++j) {
      tc::tmem_st8_splat(tb + 64u * w + 8u * j, MAGIC);
      if (!HIGH) tc::tmem_st8_splat(tb + ACC_SET1 + 64u * w + 8u * j, MAGIC);
    }
  if (NCOL == 64) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      tc::tmem_st8_splat(tb + COL_ACC_LO + 8u * j, 0u);
      tc::tmem_st8_splat(tb + COL_ACC_HI + 8u * j, 0u);
    }
  }
  tc::tmem_st_wait();
  tc::fence_before_sync();
  tc::mbar_arrive(&sh.accempty[0]);
  if (!HIGH) tc::mbar_arrive(&sh.accempty[1]);

  int64_t acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = 0;
  uint32_t ph_af = 0;  // bit s: the phase of accfull[s]
  int set = 0;      // the accumulator set of the current window (always 0 in the full form)
  uint32_t tw = tb;  // its columns
  const int ncols = min((int)a.N, NN);  // output columns actually read
  const int amode = a.alpha == 1.0 ? 0 : a.alpha == -1.0 ? 1 : 2;  // decided once, not per output
  const bool beta0 = a.beta == 0.0;
  for (Cursor c = start; c.i < c.n; c.next()) {
    if (!c.win_last()) continue;
    // lane 0 waits; the warp follows its decision (tcgen05.ld is warp-collective)
    bool ok = true;
    if (lane == 0) ok = tc::mbar_wait(&sh.accfull[set], (ph_af >> set) & 1u, WAIT_TRIES);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    ph_af ^= 1u << set;
    tw = tb + (set ? ACC_SET1 : 0u);
    if (!ok) {
      s_abort = 1;
      break;
    }
    tc::fence_after_sync();
    // 4 output columns at a time.  Padding columns (>= ncols) are never read and
    // never re-armed.
    uint32_t ra[6][4], rb[6][4];
    auto load = [&](int j, uint32_t (&r)[6][4]) {
      const uint32_t c4 = 4u * j;
      tc::tmem_ld4(tw + c4, r[0]);
      tc::tmem_ld4(tw + 64u + c4, r[1]);
      tc::tmem_ld4(tw + 128u + c4, r[2]);
      tc::tmem_ld4(tw + 192u + c4, r[3]);
      if (j >= 8) {
        tc::tmem_ld4(tb + COL_ACC_LO + c4 - 32u, r[4]);
        tc::tmem_ld4(tb + COL_ACC_HI + c4 - 32u, r[5]);
      }
    };
    auto work = [&](int j, uint32_t (&r)[6][4]) {
      const uint32_t c4 = 4u * j;
      int64_t add[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        // (G_0 * 256 + G_1) and (G_2 * 256 + G_3), each exact in 32 bits
        const int hi = (int)(r[0][i] * 256u + r[1][i] - 257u * MAGIC);
        const int lo = (int)(r[2][i] * 256u + r[3][i] - 257u * MAGIC);
        add[i] = ((int64_t)hi << 16) + (int64_t)lo;
      }
      tc::tmem_st4_splat(tw + c4, MAGIC);
      tc::tmem_st4_splat(tw + 64u + c4, MAGIC);
      tc::tmem_st4_splat(tw + 128u + c4, MAGIC);
      tc::tmem_st4_splat(tw + 192u + c4, MAGIC);
      if (j < 8) {
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[4 * j + i] += add[i];
      } else {
        uint32_t lo[4], hi[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint64_t t = (((uint64_t)r[5][i] << 32) | r[4][i]) + (uint64_t)add[i];
          lo[i] = (uint32_t)t;
          hi[i] = (uint32_t)(t >> 32);
        }
        tc::tmem_st4(tb + COL_ACC_LO + c4 - 32u, lo);
        tc::tmem_st4(tb + COL_ACC_HI + c4 - 32u, hi);
      }
    };
    if (PIPE) {
      // chunk j + 1's loads are issued right after chunk j's wait
      load(0, ra);
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (col0 + 4 * j >= ncols) break;
        tc::tmem_ld_wait();
        if (j + 1 < NJ && col0 + 4 * (j + 1) < ncols) {
          if (j & 1)
            load(j + 1, ra);
          else
            load(j + 1, rb);
        }
        if (j & 1)
          work(j, rb);
        else
          work(j, ra);
      }
    } else {
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (col0 + 4 * j >= ncols) break;
        load(j, ra);
        tc::tmem_ld_wait();
        work(j, ra);
      }
    }
    tc::tmem_st_wait();
    if (c.seg_last()) {
      const int64_t tile = c.tile;
      // the segment is the whole tile: it started at stage 0 and ends at the last
      const bool full = (c.ks + 1 == c.kst) && (c.i >= c.kst - 1);
      const int r = 32 * quarter + lane;
      const int64_t p = tile * TM + r;
      const int ep = p < a.P ? __ldg(a.xE + p) : 0;
      const int slot = (tile == first_tile) ? 0 : 1;
      double* wp = a.part + (cta * 2 + slot) * (int64_t)(NN * TM) + r;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (col0 + 4 * j >= ncols) continue;
        const uint32_t c4 = 4u * j;
        uint32_t g4[4] = {0, 0, 0, 0}, g5[4] = {0, 0, 0, 0}, g6[4] = {0, 0, 0, 0}, lo[4], hi[4];
        if (HIGH) {
          tc::tmem_ld4(tb + 256u + c4, g4);
          tc::tmem_ld4(tb + 320u + c4, g5);
          tc::tmem_ld4(tb + 384u + c4, g6);
        }
        if (j >= 8) {
          tc::tmem_ld4(tb + COL_ACC_LO + c4 - 32u, lo);
          tc::tmem_ld4(tb + COL_ACC_HI + c4 - 32u, hi);
        }
        tc::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int col = col0 + 4 * j + i;
          int64_t T;
          if (j < 8) {
            T = acc[4 * j + i];
            acc[4 * j + i] = 0;
          } else {
            T = (int64_t)(((uint64_t)hi[i] << 32) | lo[i]);
          }
          if (p < a.P && col < a.N) {
            // weights 4..6 in the units of weight 4, in FP32 (their own FP32 sums
            // carry more rounding than this), then one FP64 multiply-add onto T
            const float rest = fmaf(__uint_as_float(g6[i]), 0x1p-16f,
                                    fmaf(__uint_as_float(g5[i]), 0x1p-8f, __uint_as_float(g4[i])));
            const double sum = fma((double)rest, 0x1p-8, __ll2double_rn(T));  // units of 2^-24
            const double val = scale2(sum, ep + syE[col] - EXP_OFFSET - 24);
            if (full) {
              double* dst = a.C + p * a.csp + (int64_t)col * a.csc;
              const double av = amode == 0 ? val : amode == 1 ? -val : a.alpha * val;
              *dst = beta0 ? av : av + a.beta * (*dst);
            } else {
              wp[(int64_t)col * TM] = val;
            }
          }
        }
        if (j >= 8) {
          tc::tmem_st4_splat(tb + COL_ACC_LO + c4 - 32u, 0u);
          tc::tmem_st4_splat(tb + COL_ACC_HI + c4 - 32u, 0u);
        }
      }
      tc::tmem_st_wait();
    }
    tc::fence_before_sync();
    tc::mbar_arrive(&sh.accempty[set]);
    if (!HIGH) set ^= 1;
  }
}

template <bool TRANS>
__global__ void __launch_bounds__(NT, 1) k_ozgemm(OzArgs a) {
  if (a.skip && __ldcg(a.skip)) return;
  extern __shared__ uint8_t smem_raw[];
  __shared__ OzShared sh;
  __shared__ int sEx[2][TM];  // producers: row exponents of tiles (by tile parity)
  __shared__ volatile int s_pgo[2];  // producers: go on with iteration i (slot i % 2)
  const uint32_t raw = tc::smem_addr(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  volatile int& s_abort = sh.abort;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t G = gridDim.x, cta = blockIdx.x;
  int64_t u0, u1;
  cta_range(a, cta, G, u0, u1);
  if (u0 >= u1) return;
  const Cursor start{u0 / a.kst, (int)(u0 % a.kst), 0, u1 - u0, (int)a.kst};
  oz_setup(sh, a, NPROD + 1, NFLUSH);  // + the arrival that carries the Y bytes

  if (warp >= 4 && warp < MMA_WARP) {
    // ---------------------------------------------------------- producers
    const int pt = tid - NFLUSH, pw = pt >> 5;
    uint32_t ph_empty = 0;  // bit s: the phase of empty[s]
    // row exponents of a tile in sEx[tile % 2], written while the first stage of
    // the tile is fetched (one iteration ahead of its use, behind a named barrier)
    auto load_exps = [&](int64_t tile) {
      if (pt < TM) {
        const int64_t p = tile * TM + pt;
        sEx[tile & 1][pt] = p < a.P ? __ldg(a.xE + p) : 0;
      }
    };
    // One stage: wait for its buffer, start the Y copy, prefetch the next stage's
    // values into nxt, cut cur.  Returns false when the producers stop.
    auto stage = [&](const Cursor& c, double (&cur)[VPT], double (&nxt)[VPT]) -> bool {
      const int st = (int)(c.i % NSTAGE), slot = (int)(c.i & 1);
      // Thread 0 waits for the stage and decides whether to go on; the decision is
      // published in slot i % 2 before the named barrier and read after it, so all
      // producers leave the loop in the same iteration (slot i % 2 is next written
      // in iteration i + 2, after every producer has passed barrier i + 1).
      if (pt == 0) {
        bool go = s_abort == 0;
        if (go && c.i >= NSTAGE) go = tc::mbar_wait(&sh.empty[st], (ph_empty >> st) & 1u, WAIT_TRIES);
        if (!go) s_abort = 1;
        s_pgo[slot] = go ? 1 : 0;
      }
      if (c.i >= NSTAGE) ph_empty ^= 1u << st;
      tc::named_sync(1, NPROD);
      if (!s_pgo[slot]) return false;
      uint8_t* sA = sm + st * STAGE;
      if (pt == 0) {
        tc::mbar_arrive_expect_tx(&sh.full[st], Y_STAGE);
        tc::bulk_g2s(sA + S * A_PLANE, a.img + (int64_t)c.ks * Y_STAGE, Y_STAGE, &sh.full[st]);
      }
      if (c.i + 1 < c.n) {
        Cursor d = c;
        d.next();
        if (d.ks == 0) load_exps(d.tile);
        fetch<TRANS>(a, d.tile, d.ks, pw, lane, nxt);
      }
      cut_stage<TRANS>(cur, sEx[c.tile & 1], sA, pw, lane);
      tc::fence_async_smem();
      tc::mbar_arrive(&sh.full[st]);
      return true;
    };
    double va[VPT], vb[VPT];
    Cursor c = start;
    load_exps(c.tile);
    fetch<TRANS>(a, c.tile, c.ks, pw, lane, va);
    // two stages per trip, so that the two value buffers swap roles without copies
    while (c.i < c.n) {
      if (!stage(c, va, vb)) break;
      c.next();
      if (c.i >= c.n) break;
      if (!stage(c, vb, va)) break;
      c.next();
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) oz_mma_role<true>(sh, start, sm);
    __syncwarp();
  } else if (warp < 4) {
    oz_flush_role<false, true, 4>(sh, a, start, cta);
  }
  oz_teardown(sh, a);
}

// The same product with op(X) already cut: img holds, per (tile, stage), the
// seven digit planes in the stage layout (A_PLANE bytes each, contiguous), so a
// stage is two bulk copies issued by one thread.  Warps 0..7 flush, warp 8
// copies, warp 9 issues the MMAs.
constexpr int NFLUSH_IMG = 256;  // eight flush warps, 32 output columns each
constexpr int NT_IMG = NFLUSH_IMG + 64;

// LOW: the reduced form -- only digits 0..3 of A and of Y are copied and multiplied
// (the 10 pairs of weight <= 3, all summed exactly): error ~2^-30 of max|x| max|y|.
template <bool LOW, bool YD1>
__global__ void __launch_bounds__(NT_IMG, 1) k_ozgemm_img(OzArgs a, const uint8_t* __restrict__ ximg) {
  constexpr int SUSE = LOW ? 4 : S;   // digit planes of X used
  constexpr int YUSE = YD1 ? 1 : SUSE;  // digit planes of Y copied
  extern __shared__ uint8_t smem_raw[];
  __shared__ OzShared sh;
  const uint32_t raw = tc::smem_addr(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  volatile int& s_abort = sh.abort;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t G = gridDim.x, cta = blockIdx.x;
  int64_t u0, u1;
  cta_range(a, cta, G, u0, u1);
  if (u0 >= u1) return;
  const Cursor start{u0 / a.kst, (int)(u0 % a.kst), 0, u1 - u0, (int)a.kst};
  oz_setup(sh, a, 1, NFLUSH_IMG);

  if (warp == 8) {
    if (lane == 0) {
      uint32_t ph_empty = 0;  // bit s: the phase of empty[s]
      for (Cursor c = start; c.i < c.n; c.next()) {
        const int st = (int)(c.i % NSTAGE);
        if (c.i >= NSTAGE) {
          if (s_abort || !tc::mbar_wait(&sh.empty[st], (ph_empty >> st) & 1u, WAIT_TRIES)) {
            s_abort = 1;
            break;
          }
          ph_empty ^= 1u << st;
        }
        uint8_t* sA = sm + st * STAGE;
        tc::mbar_arrive_expect_tx(&sh.full[st], SUSE * A_PLANE + YUSE * Y_PLANE);
        tc::bulk_g2s(sA, ximg + (c.tile * a.kst + c.ks) * (int64_t)(S * A_PLANE), SUSE * A_PLANE,
                     &sh.full[st]);
        tc::bulk_g2s(sA + S * A_PLANE, a.img + (int64_t)c.ks * Y_STAGE, YUSE * Y_PLANE, &sh.full[st]);
      }
    }
    __syncwarp();
  } else if (warp == 9) {
    if (lane == 0) oz_mma_role<!LOW, YD1>(sh, start, sm);
    __syncwarp();
  } else {
    oz_flush_role<true, !LOW, 8>(sh, a, start, cta);
  }
  oz_teardown(sh, a);
}

// Cut op(X) into its digit image (the stage layout of k_ozgemm_img): one CTA of
// NPROD threads per (tile, stage) unit, grid-stride.
// sqpart (when given): sqpart[blockIdx.x] = the sum of the squares of the values
// the CTA cut (FP64 multiply-adds), so that the partials summed in order give
// ||X||_F^2 from the same read of X (the FP64 pipe is otherwise idle in this
// kernel).  A thread sums each unit's values, then 32 unit sums, then those
// block sums: no chain of additions is longer than ~32 terms (one running sum
// over the ~8000 values a thread cuts at 60000 x 20000 loses ~40 units of
// 2^-53), then the CTA's threads in a fixed-order tree.
template <bool TRANS, typename E>
__global__ void __launch_bounds__(NPROD) k_oz_xcut(OzArgs a, uint8_t* __restrict__ ximg,
                                                   double* __restrict__ sqpart) {
  __shared__ int sE[TM];
  __shared__ double sred[NPROD / 32];
  const int pw = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t T = a.tiles * a.kst;
  int64_t prev_tile = -1;
  double qt = 0.0, qb = 0.0;  // the thread's total and its current block of units
  int nq = 0;                 // unit sums in qb
  for (int64_t u = blockIdx.x; u < T; u += gridDim.x) {
    const int64_t tile = u / a.kst;
    const int ks = (int)(u % a.kst);
    if (tile != prev_tile) {
      __syncthreads();
      if (threadIdx.x < TM) {
        const int64_t p = tile * TM + threadIdx.x;
        sE[threadIdx.x] = p < a.P ? __ldg(a.xE + p) : 0;
      }
      __syncthreads();
      prev_tile = tile;
    }
    double v[VPT];
    fetch<TRANS, E>(a, tile, ks, pw, lane, v);
    cut_stage<TRANS>(v, sE, ximg + u * (int64_t)(S * A_PLANE), pw, lane);
    if (sqpart) {
      double su = 0.0;
#pragma unroll
      for (int i = 0; i < VPT; ++i) su = fma(v[i], v[i], su);
      qb += su;
      if (++nq == 32) {
        qt += qb;
        qb = 0.0;
        nq = 0;
      }
    }
  }
  if (sqpart) {
    double q = qt + qb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_down_sync(0xffffffffu, q, o);
    if (lane == 0) sred[pw] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < NPROD / 32; ++w) t += sred[w];
      sqpart[blockIdx.x] = t;
    }
  }
}

// Combine the partial tiles of tiles split across CTAs, in a fixed order.  Grid:
// (tiles, ceil(TM N LANES / 256)); the elements of tile t (rows_t x N of them,
// row index fastest) are numbered densely and each CTA takes 256 / LANES of them
// with LANES threads per element: thread l sums the partials of the contributing
// CTAs cf + l, cf + l + LANES, ... in CTA order (four running sums, so that four
// loads are in flight, combined in a fixed order; one sum when LANES = 1), and
// the LANES sums are added in lane order.  Tile t is covered by CTAs cf..cl; every one of them but cf
// starts its range inside t, so t is its first tile (slot 0); cf holds t in slot
// 1 unless its range also starts inside t.  CTAs with an empty range (more CTAs
// than units) wrote nothing and are skipped.
//
// CTA c's range starts at floor(c T / G), so the owner of unit u (the last CTA
// whose range starts at or before u) is floor(((u + 1) G - 1) / T), and cf's
// range starts inside t exactly when cf T >= t kst G.  The owner is estimated in
// FP32 and corrected with exact integer products (no 64-bit division).
__device__ __forceinline__ int64_t oz_owner(int64_t u, int64_t T, int64_t G) {
  const int64_t x = (u + 1) * G - 1;
  int64_t c = (int64_t)((float)x / (float)T);
  while (c > 0 && c * T > x) --c;
  while ((c + 1) * T <= x) ++c;
  return c;
}

// One CTA's share of the fixup: NTHR threads, LANES per element.  Returns early
// (the whole CTA alike) when it has nothing to sum.
template <int LANES, int NTHR>
__device__ __forceinline__ void oz_fixup_cta(const OzArgs& a, int G) {
  constexpr int ELEMS = NTHR / LANES;
  __shared__ int64_t s_cf, s_cl;
  __shared__ int s_slot_f;
  const int64_t t = blockIdx.x;
  const int64_t T = a.tiles * a.kst;
  const int rows_t = (int)min((int64_t)TM, a.P - t * TM);
  const int nel = rows_t * (int)min(a.N, (int64_t)NN);
  if ((int)blockIdx.y * ELEMS >= nel) return;  // the whole CTA
  if (threadIdx.x == 0) {
    const int64_t cf = oz_owner(t * a.kst, T, G);
    s_cf = cf;
    s_cl = oz_owner((t + 1) * a.kst - 1, T, G);
    s_slot_f = (cf * T >= t * a.kst * G) ? 0 : 1;
  }
  __syncthreads();
  const int64_t cf = s_cf, cl = s_cl;
  if (cf == cl) return;
  const int slot_f = s_slot_f;
  const int lane = threadIdx.x % LANES;
  const int e = blockIdx.y * ELEMS + threadIdx.x / LANES;
  const bool valid = e < nel;  // the same in the LANES threads of an element
  const int c = valid ? e / rows_t : 0, r = valid ? e - c * rows_t : 0;
  const int64_t p = t * TM + r;
  const double* src = a.part + (int64_t)c * TM + r;
  const bool all_nonempty = T >= G;  // then every CTA's range holds a unit
  auto part = [&](int64_t q) -> double {
    const int slot = (q == cf) ? slot_f : 0;
    return (all_nonempty || q * T / G < (q + 1) * T / G) ? src[(q * 2 + slot) * (int64_t)(NN * TM)]
                                                          : 0.0;
  };
  double s = 0.0;
  if (valid && LANES == 1) {
    // a few partials: one running sum (the FP64 pipe, not memory, limits this case)
    s = part(cf);
    for (int64_t q = cf + 1; q <= cl; ++q) s += part(q);
  } else if (valid) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t q = cf + lane;
    for (; q + 3 * LANES <= cl; q += 4 * LANES) {
      const double v0 = part(q), v1 = part(q + LANES), v2 = part(q + 2 * LANES), v3 = part(q + 3 * LANES);
      s0 += v0;
      s1 += v1;
      s2 += v2;
      s3 += v3;
    }
    if (q <= cl) s0 += part(q);  // fewer than four left
    if (q + LANES <= cl) s1 += part(q + LANES);
    if (q + 2 * LANES <= cl) s2 += part(q + 2 * LANES);
    s = (s0 + s1) + (s2 + s3);
  }
  // lanes of one element are adjacent threads of one warp
#pragma unroll
  for (int o = 1; o < LANES; o <<= 1) {
    const double other = __shfl_down_sync(0xffffffffu, s, o, LANES);
    if ((lane & (2 * o - 1)) == 0) s += other;
  }
  if (lane == 0 && valid) {
    double* dst = a.C + p * a.csp + (int64_t)c * a.csc;
    const double as = (a.alpha == 1.0) ? s : a.alpha * s;
    *dst = (a.beta == 0.0) ? as : as + a.beta * (*dst);
  }
}

template <int LANES>
__global__ void __launch_bounds__(256, 6) k_oz_fixup(OzArgs a, int G) {
  if (a.skip && __ldcg(a.skip)) return;
  oz_fixup_cta<LANES, 256>(a, G);
}

// The fused Gram + Cholesky (the b x b Gram S = X^T X of CholQR, Alg. 1's Z = Y^T Y
// in QB form): the fixup of the split Gram, then the CTA that finishes last -- the
// one whose increment of the launch's arrival counter completes it -- factors S
// (chol.cuh) and resets the counter for the next launch.  Writers publish S with
// a fence before their arrival; the last CTA reads it after its own fence, with
// loads that bypass L1.  Nothing waits on another CTA.
__global__ void __launch_bounds__(CHOL_NT) k_oz_fixup_chol(OzArgs a, int G, CholJob job) {
  __shared__ int s_last;
  oz_fixup_cta<16, CHOL_NT>(a, G);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(job.count, 1) == (int)(gridDim.x * gridDim.y) - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  chol_inv_cta(a.C, (int)a.N, job.tau, job.Rinv, a.flags, job.dead, job.near);
  if (threadIdx.x == 0) *job.count = 0;
}

// The fixup launch: lanes per element by the number of CTAs that share a tile
// (about G kst / T + 1): one up to eight sharers, four up to 64, sixteen beyond.
cudaError_t launch_fixup(const OzArgs& a, int G, cudaStream_t st) {
  const int64_t T = a.tiles * a.kst;
  const int64_t elems = (int64_t)TM * std::min<int64_t>(a.N, NN);
  const int64_t sharers = (int64_t)G * a.kst / std::max<int64_t>(T, 1) + 1;
  if (sharers <= 8) {
    k_oz_fixup<1><<<dim3((unsigned)a.tiles, (unsigned)((elems + 255) / 256)), 256, 0, st>>>(a, G);
  } else if (sharers <= 64) {
    k_oz_fixup<4><<<dim3((unsigned)a.tiles, (unsigned)((elems * 4 + 255) / 256)), 256, 0, st>>>(a, G);
  } else {
    k_oz_fixup<16><<<dim3((unsigned)a.tiles, (unsigned)((elems * 16 + 255) / 256)), 256, 0, st>>>(a, G);
  }
  return launched();
}

cudaError_t oz_rowcol_exponents(const double* X, int64_t ld, int64_t rows, int64_t cols,
                                int* rowE, int* colE, cudaStream_t st, bool accumulate_rows,
                                const int* skip) {
  if (colE) {
    cudaError_t e = colmaxexp(X, ld, rows, cols, colE, st, skip);
    if (e != cudaSuccess) return e;
  }
  if (rowE) {
    const int64_t csplit = cols >= 256 ? 16 : 1;
    const bool direct = csplit == 1 && !accumulate_rows;
    if (skip && !direct) return cudaErrorInvalidValue;
    if (!accumulate_rows && !direct) {
      cudaError_t e = cudaMemsetAsync(rowE, 0, rows * sizeof(int), st);
      if (e != cudaSuccess) return e;
    }
    const int64_t cchunk = (cols + csplit - 1) / csplit;
    dim3 grid((unsigned)((rows + 255) / 256), (unsigned)((cols + cchunk - 1) / cchunk));
    k_oz_rowmaxexp<<<grid, 256, 0, st>>>(X, ld, rows, cols, cchunk, rowE, direct, skip);
    return launched();
  }
  return cudaSuccess;
}

namespace {
OzArgs make_args(int64_t P, int64_t N, int64_t K, double alpha, const double* X, int64_t ldx,
                 const int* xE, double beta, GemmOut out, const OzWorkspace& w, int* flags) {
  OzArgs a;
  a.P = P;
  a.K = K;
  a.N = N;
  a.X = X;
  a.X32 = nullptr;
  a.ldx = ldx;
  a.xE = xE;
  a.yE = w.yE;
  a.img = w.img;
  a.alpha = alpha;
  a.beta = beta;
  a.C = out.C;
  a.csp = out.csp;
  a.csc = out.csc;
  a.part = w.part;
  a.tiles = (P + TM - 1) / TM;
  a.kst = (K + KS - 1) / KS;
  a.flags = flags;
  a.vec = X && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (ldx % 2 == 0);
  // short tiles (K <= 64): whole tiles per CTA beat splitting plus a fixup; long
  // tiles are split along K (stream-K), also when there are few of them
  a.whole_tiles = a.kst <= 4;
  a.skip = nullptr;
  return a;
}

// Y's exponents and digit image (shared by both GEMM kernels).
// yE_known: Y's column exponents when the caller has them (else computed into w.yE).
cudaError_t prepare_y(const double* Y, int64_t ldy, int64_t K, int64_t N, const OzWorkspace& w,
                      const int* yE_known, cudaStream_t st, const int* skip = nullptr) {
  const int64_t kst = (K + KS - 1) / KS;
  const int* yE = yE_known;
  if (!yE) {
    cudaError_t e = colmaxexp(Y, ldy, K, N, w.yE, st, skip);
    if (e != cudaSuccess) return e;
    yE = w.yE;
  }
  const int64_t ythreads = kst * NN * 2;
  k_oz_ycut<<<(unsigned)((ythreads + 255) / 256), 256, 0, st>>>(Y, ldy, K, (int)N, yE, w.img, kst,
                                                                  skip);
  return launched();
}

template <typename F>
cudaError_t set_smem_once(F kernel, std::atomic<bool>& done) {
  if (done.load(std::memory_order_acquire)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_DYN);
  if (e == cudaSuccess) done.store(true, std::memory_order_release);
  return e;
}
}  // namespace

cudaError_t oz_prepare() {
  // set once per process; concurrent first calls set the same attribute twice
  static std::atomic<bool> a0{false}, a1{false}, a2{false}, a3{false}, a4{false}, a5{false};
  cudaError_t e = set_smem_once(k_ozgemm<false>, a0);
  if (e == cudaSuccess) e = set_smem_once(k_ozgemm<true>, a1);
  if (e == cudaSuccess) e = set_smem_once(k_ozgemm_img<false, false>, a2);
  if (e == cudaSuccess) e = set_smem_once(k_ozgemm_img<true, false>, a3);
  if (e == cudaSuccess) e = set_smem_once(k_ozgemm_img<false, true>, a4);
  if (e == cudaSuccess) e = set_smem_once(k_ozgemm_img<true, true>, a5);
  return e;
}

int64_t oz_ximg_bytes(int64_t P, int64_t K) {
  return ((P + TM - 1) / TM) * ((K + KS - 1) / KS) * (int64_t)(S * A_PLANE);
}

int oz_cut_ctas(int64_t P, int64_t K, int ctas) {
  const int64_t units = ((P + TM - 1) / TM) * ((K + KS - 1) / KS);
  return (int)std::min<int64_t>(units, (int64_t)ctas * 4);
}

cudaError_t oz_cut_x(bool trans, int64_t P, int64_t K, const void* X, int dtype, int64_t ldx,
                     const int* xE, uint8_t* ximg, int ctas, cudaStream_t st, double* sqpart) {
  if (P <= 0 || K <= 0) return cudaSuccess;
  OzWorkspace none{};
  const bool f32 = dtype == LRA_F32;
  OzArgs a = make_args(P, 1, K, 1.0, f32 ? nullptr : (const double*)X, ldx, xE, 0.0,
                       GemmOut{nullptr, 0, 0}, none, nullptr);
  if (f32) {
    a.X32 = (const float*)X;
    a.vec = ((reinterpret_cast<uintptr_t>(X) & 7) == 0) && (ldx % 2 == 0);
  }
  const unsigned grid = (unsigned)oz_cut_ctas(P, K, ctas);
  if (f32) {
    if (trans)
      k_oz_xcut<true, float><<<grid, NPROD, 0, st>>>(a, ximg, sqpart);
    else
      k_oz_xcut<false, float><<<grid, NPROD, 0, st>>>(a, ximg, sqpart);
  } else {
    if (trans)
      k_oz_xcut<true, double><<<grid, NPROD, 0, st>>>(a, ximg, sqpart);
    else
      k_oz_xcut<false, double><<<grid, NPROD, 0, st>>>(a, ximg, sqpart);
  }
  return launched();
}

cudaError_t ozgemm_img(int64_t P, int64_t N, int64_t K, double alpha, const uint8_t* ximg,
                       const int* xE, const double* Y, int64_t ldy, double beta, GemmOut out,
                       const OzWorkspace& w, int* flags, cudaStream_t st, bool low, bool ydig1) {
  if (P <= 0 || N <= 0) return cudaSuccess;
  if (N > NN || K <= 0 || K > MAX_K) return cudaErrorInvalidValue;
  if (oz_img_bytes(K) > w.img_bytes) return cudaErrorInvalidValue;
  cudaError_t e = oz_prepare();
  if (e != cudaSuccess) return e;
  e = prepare_y(Y, ldy, K, N, w, nullptr, st);
  if (e != cudaSuccess) return e;
  OzArgs a = make_args(P, N, K, alpha, nullptr, 0, xE, beta, out, w, flags);
  const int G = w.ctas;
  if (low && ydig1)
    k_ozgemm_img<true, true><<<G, NT_IMG, SMEM_DYN, st>>>(a, ximg);
  else if (low)
    k_ozgemm_img<true, false><<<G, NT_IMG, SMEM_DYN, st>>>(a, ximg);
  else if (ydig1)
    k_ozgemm_img<false, true><<<G, NT_IMG, SMEM_DYN, st>>>(a, ximg);
  else
    k_ozgemm_img<false, false><<<G, NT_IMG, SMEM_DYN, st>>>(a, ximg);
  e = launched();
  if (e != cudaSuccess || a.whole_tiles) return e;
  return launch_fixup(a, G, st);
}

cudaError_t ozgemm(bool trans, int64_t P, int64_t N, int64_t K, double alpha, const double* X,
                   int64_t ldx, const int* xE, const double* Y, int64_t ldy, double beta, GemmOut out,
                   const OzWorkspace& w, int* flags, cudaStream_t st, const int* yE_known,
                   const CholJob* chol, const int* skip) {
  if (P <= 0 || N <= 0) return cudaSuccess;
  if (N > NN || K <= 0 || K > MAX_K) return cudaErrorInvalidValue;
  if (oz_img_bytes(K) > w.img_bytes) return cudaErrorInvalidValue;
  // a skipped product leaves nothing for a Cholesky to read
  if (skip && chol) return cudaErrorInvalidValue;
  cudaError_t e = oz_prepare();
  if (e != cudaSuccess) return e;
  e = prepare_y(Y, ldy, K, N, w, yE_known, st, skip);
  if (e != cudaSuccess) return e;
  OzArgs a = make_args(P, N, K, alpha, X, ldx, xE, beta, out, w, flags);
  if (yE_known) a.yE = yE_known;
  a.skip = skip;
  const int G = w.ctas;
  if (trans)
    k_ozgemm<true><<<G, NT, SMEM_DYN, st>>>(a);
  else
    k_ozgemm<false><<<G, NT, SMEM_DYN, st>>>(a);
  e = launched();
  if (e != cudaSuccess) return e;
  if (chol) {
    // the product is the b x b Gram (P = N = b <= 64, C with ld b): factor it
    if (a.whole_tiles)
      return chol_inv(out.C, (int)N, chol->tau, chol->Rinv, flags, st, chol->dead, chol->near);
    const int64_t elems = (int64_t)P * N;
    k_oz_fixup_chol<<<dim3(1, (unsigned)((elems * 16 + CHOL_NT - 1) / CHOL_NT)), CHOL_NT, 0, st>>>(a, G, *chol);
    return launched();
  }
  if (a.whole_tiles) return e;
  return launch_fixup(a, G, st);
}

}  // namespace lra
