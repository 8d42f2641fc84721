// FP64-accurate skinny GEMM on the tcgen05 tensor cores: C = alpha op(X) Y + beta C
// with X, Y, C in FP64 and N <= 64.  These are the full passes over A of the
// farPCA block (arxiv 2506.03859 Alg. 1 steps A^T(A G_j), A G_j, A^T Y_j).
//
// GB300's FP64 pipe delivers about 1.2 TFLOP/s, while such a pass streams A once
// from HBM: run as FP64 FMAs it is ~60x slower than the memory bound.  Instead
// every operand is cut, error-free, into bf16 slices (the splitting idea of
// Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 2012):
//
//   each row p of op(X) is scaled by 2^-e_p (|x| < 2^e_p over the row) and
//   each column c of Y by 2^-f_c; the scaled value, truncated to a 56-bit fixed
//   point number, is x = 2^-7 sum_{s<8} v_s with v_s = d_s 2^(-7 s),
//   d_s in [0, 127] carrying the sign of x.  Every v_s is exact in bf16.
//
//   x y = 2^-14 sum_{s,t} v_s w_t; the 36 pairs with s + t <= 7 are kept (the
//   rest is below 2^-56 relative), each a bf16 MMA on the tensor core with FP32
//   accumulation in TMEM.  The pairs of weight w = s + t <= 4 are summed per
//   weight over windows of 32 values of K: every such sum is an integer
//   multiple of 2^(-7 w) below 2^22 units (at most 5 pairs x 32 x 127^2), so the
//   FP32 accumulator holds it exactly and adding 1.5 * 2^23 turns it into an
//   integer.  The five integers are combined into one int64 per output in units
//   of 2^-28 (exact).  The pairs of weight >= 5 (at most 2^-35 of a product) run
//   in one FP32 accumulator over all of K.  The tile is then (int64 * 2^-28 +
//   fp32) * 2^(e_p + f_c - 2058), written in FP64.  Against exact dot products
//   the error is that of an FP64 GEMM (2^-52 of |op(X)| |Y| on Gaussian data).
//
// Work split: one CTA per SM walks a contiguous range of (row tile, 32-deep
// window) units ("stream-K"); tiles whose windows span two or more CTAs are
// written as partial sums and combined by a fixup kernel in a fixed order.
// Inside a CTA the work is pipelined by warp role: eight producer warps load
// a 128 x 32 block of op(X) from HBM, slice it into 8 bf16 planes of a shared
// memory stage (two stages, K-major core-matrix layout) and copy the pre-sliced
// 64 x 32 block of Y; one thread issues the window's 72 MMAs; four warps flush
// the exact sums from TMEM and write the tile.  mbarriers hand stages and the
// TMEM accumulators between the roles; every wait is bounded.
#include <math.h>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace lra {

namespace {
constexpr int S = 8;               // slices per operand (7 bits each)
constexpr int BETA = 7;            // bits per slice
constexpr int TM = 128;            // rows of op(X) per tile
constexpr int KW = 32;             // K per window (one pipeline stage)
constexpr int NN = 64;             // output columns (N padded)
constexpr int NPROD = 256;         // producer threads (warps 4..11)
constexpr int NFLUSH = 128;        // flush threads (warps 0..3)
constexpr int NT = NFLUSH + NPROD + 32;  // + one MMA warp (warp 12)
constexpr int A_PLANE = TM * KW * 2;     // bytes of one slice plane of the op(X) block
constexpr int Y_PLANE = NN * KW * 2;     // bytes of one slice plane of the Y block
constexpr int STAGE = S * (A_PLANE + Y_PLANE);
constexpr int NSTAGE = 2;
constexpr int SMEM_DYN = NSTAGE * STAGE + 1024;
constexpr uint32_t LBO = 128, SBO = 512;         // core-matrix strides (K, rows)
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t COL_G5 = 320;                  // FP32 sum of the pairs of weight >= 5
constexpr uint32_t COL_ACC_LO = 384, COL_ACC_HI = 448;  // int64 exact sum, two words
constexpr int EXACT_GROUPS = 5;                   // weights 0..4, TMEM columns 64 w
constexpr long WAIT_TRIES = 1L << 22;
constexpr int EXP_OFFSET = 2058;  // 2 * 1022 + 2 * BETA: see the scaling above
}  // namespace

int64_t oz_img_bytes(int64_t K) { return (K + KW - 1) / KW * S * Y_PLANE; }
int64_t oz_part_elems(int ctas) { return (int64_t)ctas * 2 * TM * NN; }

// Offset of element (row, k), k < 32, in the K-major core-matrix layout of a
// stage plane: core (row/8, k/8) at ((row/8)*4 + k/8)*128, row-major inside.
__host__ __device__ __forceinline__ uint32_t core_offset(uint32_t row, uint32_t k) {
  return (((row >> 3) << 2) + (k >> 3)) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

// |a| as a 56-bit fixed-point integer relative to 2^(emax - 1022) (emax = the
// largest biased exponent of the row/column), and its sign.
__device__ __forceinline__ uint64_t fixed56(double a, int emax, uint32_t& sign) {
  const uint64_t bits = (uint64_t)__double_as_longlong(a);
  sign = (uint32_t)(bits >> 63);
  const int E = (int)((bits >> 52) & 0x7FFu);
  const uint64_t M = (E != 0) ? ((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : 0ull;
  const int d = emax - E;  // >= 0 by the choice of emax
  if (d <= 3) return M << (3 - d);
  const int sh = d - 3;
  return sh < 64 ? (M >> sh) : 0ull;
}

// bf16 bits of d * 2^(-7 s) (d < 128, exact), sign in bit 15.
template <int SLICE>
__device__ __forceinline__ uint32_t slice_bf16(uint64_t x, uint32_t sign) {
  const uint32_t d = (uint32_t)(x >> (BETA * (S - 1 - SLICE))) & 0x7Fu;
  constexpr float sc = (SLICE == 0) ? 1.0f : (SLICE == 1) ? 0x1p-7f : (SLICE == 2) ? 0x1p-14f
                       : (SLICE == 3) ? 0x1p-21f : (SLICE == 4) ? 0x1p-28f : (SLICE == 5) ? 0x1p-35f
                       : (SLICE == 6) ? 0x1p-42f : 0x1p-49f;
  const float f = __fmaf_rn(__int_as_float(0x4B000000 | (int)d), sc, -8388608.0f * sc);
  return (__float_as_uint(f) >> 16) | (sign << 15);
}

template <int SLICE>
__device__ __forceinline__ uint32_t pack2(uint64_t x0, uint32_t s0, uint64_t x1, uint32_t s1) {
  return slice_bf16<SLICE>(x0, s0) | (slice_bf16<SLICE>(x1, s1) << 16);
}

// ---------------------------------------------------------------- prep kernels

// out[c] = largest biased exponent of X[:, c] (one CTA per column).
__global__ void __launch_bounds__(256) k_oz_colmaxexp(const double* __restrict__ X, int64_t ld,
                                                      int64_t rows, int* __restrict__ out) {
  __shared__ int red[8];
  const int64_t c = blockIdx.x;
  int e = 0;
  for (int64_t i = threadIdx.x; i < rows; i += 256) {
    const uint64_t b = (uint64_t)__double_as_longlong(__ldg(X + i + c * ld));
    e = max(e, (int)((b >> 52) & 0x7FFu));
  }
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_down_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int q = 0; q < 8; ++q) t = max(t, red[q]);
    out[c] = t;
  }
}

// out[r] = max over the columns of X[r, :] of the biased exponent (out pre-zeroed).
__global__ void __launch_bounds__(256) k_oz_rowmaxexp(const double* __restrict__ X, int64_t ld,
                                                      int64_t rows, int64_t cols, int64_t cchunk,
                                                      int* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (r >= rows) return;
  const int64_t c0 = (int64_t)blockIdx.y * cchunk;
  const int64_t c1 = (c0 + cchunk < cols) ? c0 + cchunk : cols;
  int e = 0;
  for (int64_t c = c0; c < c1; ++c) {
    const uint64_t b = (uint64_t)__double_as_longlong(__ldg(X + r + c * ld));
    e = max(e, (int)((b >> 52) & 0x7FFu));
  }
  atomicMax(out + r, e);
}

// Pre-sliced Y: img[w][s] is the 64 x 32 (N x K) bf16 block of slice s of
// window w in the core-matrix layout.  One thread per (window, column c, 8-wide
// k chunk j).
__global__ void __launch_bounds__(256) k_oz_yslice(const double* __restrict__ Y, int64_t ldy,
                                                   int64_t K, int N, const int* __restrict__ yE,
                                                   uint8_t* __restrict__ img, int64_t kwins) {
  const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (idx >= kwins * NN * 4) return;
  const int j = (int)(idx & 3);
  const int c = (int)((idx >> 2) & (NN - 1));
  const int64_t w = idx >> 8;
  const int emax = c < N ? yE[c] : 0;
  uint64_t x[8];
  uint32_t sg[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t k = w * KW + 8 * j + i;
    const double v = (c < N && k < K) ? __ldg(Y + k + (int64_t)c * ldy) : 0.0;
    x[i] = fixed56(v, emax, sg[i]);
  }
  uint8_t* base = img + (w * S) * Y_PLANE + core_offset((uint32_t)c, (uint32_t)(8 * j));
#define LRA_YS(SL)                                                                          \
  {                                                                                         \
    uint4 q;                                                                                \
    q.x = pack2<SL>(x[0], sg[0], x[1], sg[1]);                                              \
    q.y = pack2<SL>(x[2], sg[2], x[3], sg[3]);                                              \
    q.z = pack2<SL>(x[4], sg[4], x[5], sg[5]);                                              \
    q.w = pack2<SL>(x[6], sg[6], x[7], sg[7]);                                              \
    *reinterpret_cast<uint4*>(base + (SL)*Y_PLANE) = q;                                     \
  }
  LRA_YS(0) LRA_YS(1) LRA_YS(2) LRA_YS(3) LRA_YS(4) LRA_YS(5) LRA_YS(6) LRA_YS(7)
#undef LRA_YS
}

// ---------------------------------------------------------------- main kernel

struct OzArgs {
  int64_t P, K, N;
  const double* X;
  int64_t ldx;
  const int* xE;       // biased max exponent of each row of op(X)
  const int* yE;       // biased max exponent of each column of Y
  const uint8_t* img;  // pre-sliced Y
  double alpha, beta;
  double* C;
  int64_t csp, csc;
  double* part;        // [cta][2][TM][NN] partial tiles
  int64_t tiles, kwins;
  int* flags;
  bool vec;            // 16-byte loads allowed (trans layout)
};

// Producer: slice the 128 x 32 block (tile, window w) of op(X) into the eight
// planes of a stage.  pt = producer thread 0..255.
template <bool TRANS>
__device__ __forceinline__ void slice_window(const OzArgs& a, int64_t tile, int64_t w,
                                             uint8_t* sA, const int* sE, int pt) {
  const int lane = pt & 31, pw = pt >> 5;
  const int64_t p0 = tile * TM, k0 = w * KW;
  if (TRANS) {
    // op(X)[p, k] = X[k + p*ldx]: each warp instruction covers one core matrix
    // (8 rows x 8 k): lane -> row r8 = lane & 7, k pair q = lane >> 3.
    const int r8 = lane & 7, q = lane >> 3;
    double v0[8], v1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int core = pw + 8 * i, rg = core >> 2, kc = core & 3;
      const int64_t p = p0 + rg * 8 + r8, k = k0 + kc * 8 + 2 * q;
      v0[i] = 0.0;
      v1[i] = 0.0;
      if (p < a.P) {
        const double* src = a.X + k + p * a.ldx;
        if (a.vec && k + 1 < a.K) {
          const double2 t = __ldg(reinterpret_cast<const double2*>(src));
          v0[i] = t.x;
          v1[i] = t.y;
        } else {
          if (k < a.K) v0[i] = __ldg(src);
          if (k + 1 < a.K) v1[i] = __ldg(src + 1);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int core = pw + 8 * i, rg = core >> 2, kc = core & 3;
      const int row = rg * 8 + r8;
      const int emax = sE[row];
      uint32_t s0, s1;
      const uint64_t x0 = fixed56(v0[i], emax, s0), x1 = fixed56(v1[i], emax, s1);
      uint8_t* dst = sA + core * 128 + r8 * 16 + q * 4;
#define LRA_XT(SL) *reinterpret_cast<uint32_t*>(dst + (SL)*A_PLANE) = pack2<SL>(x0, s0, x1, s1);
      LRA_XT(0) LRA_XT(1) LRA_XT(2) LRA_XT(3) LRA_XT(4) LRA_XT(5) LRA_XT(6) LRA_XT(7)
#undef LRA_XT
      (void)kc;
    }
  } else {
    // op(X)[p, k] = X[p + k*ldx]: lanes along rows, each thread 8 consecutive k.
    const int rgrp = pw & 3, kc0 = (pw >> 2) * 2;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int row = rgrp * 32 + lane, kc = kc0 + h;
      const int64_t p = p0 + row, kb = k0 + kc * 8;
      double v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        v[i] = (p < a.P && kb + i < a.K) ? __ldg(a.X + p + (kb + i) * a.ldx) : 0.0;
      const int emax = sE[row];
      uint64_t x[8];
      uint32_t sg[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fixed56(v[i], emax, sg[i]);
      uint8_t* dst = sA + core_offset((uint32_t)row, (uint32_t)(kc * 8));
#define LRA_XS(SL)                                                \
  {                                                               \
    uint4 q;                                                      \
    q.x = pack2<SL>(x[0], sg[0], x[1], sg[1]);                    \
    q.y = pack2<SL>(x[2], sg[2], x[3], sg[3]);                    \
    q.z = pack2<SL>(x[4], sg[4], x[5], sg[5]);                    \
    q.w = pack2<SL>(x[6], sg[6], x[7], sg[7]);                    \
    *reinterpret_cast<uint4*>(dst + (SL)*A_PLANE) = q;            \
  }
      LRA_XS(0) LRA_XS(1) LRA_XS(2) LRA_XS(3) LRA_XS(4) LRA_XS(5) LRA_XS(6) LRA_XS(7)
#undef LRA_XS
    }
  }
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// An FP32 value that is an integer multiple n of 2^-k with |n| < 2^22, as n:
// adding 1.5 * 2^23 after scaling by 2^k puts n in the low mantissa bits.
__device__ __forceinline__ int exact_int(uint32_t bits, float scale) {
  return __float_as_int(__fmaf_rn(__uint_as_float(bits), scale, 12582912.0f)) - 0x4B400000;
}

// The CTA's windows: a contiguous range [u0, u1) of (tile, window) units, tile-major.
struct Walk {
  int64_t u0, u1, kwins;
  __device__ __forceinline__ int64_t tile(int64_t u) const { return u / kwins; }
  __device__ __forceinline__ bool seg_first(int64_t u) const { return u == u0 || u % kwins == 0; }
  __device__ __forceinline__ bool seg_last(int64_t u) const {
    return u + 1 == u1 || (u + 1) % kwins == 0;
  }
};

template <bool TRANS>
__global__ void __launch_bounds__(NT, 1) k_ozgemm(OzArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_accfull, bar_accempty;
  __shared__ int sEp[TM];  // producers: row exponents of the current tile
  __shared__ int syE[NN];
  __shared__ volatile int s_abort;
  const uint32_t raw = tc::smem_addr(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t T = a.tiles * a.kwins;
  const int64_t G = gridDim.x, cta = blockIdx.x;
  const Walk wk{cta * T / G, (cta + 1) * T / G, a.kwins};
  if (wk.u0 >= wk.u1) return;

  if (warp == 0) tc::tmem_alloc(&s_tmem, TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      tc::mbar_init(&bar_full[s], NPROD);
      tc::mbar_init(&bar_empty[s], 1);
    }
    tc::mbar_init(&bar_accfull, 1);
    tc::mbar_init(&bar_accempty, NFLUSH);
    s_abort = 0;
  }
  if (tid < NN) syE[tid] = tid < a.N ? a.yE[tid] : 0;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const int64_t first_tile = wk.tile(wk.u0);

  if (warp >= 4 && warp < 12) {
    // ---------------------------------------------------------- producers
    const int pt = tid - NFLUSH;
    uint32_t ph_empty[NSTAGE] = {0, 0};
    int64_t cur_tile = -1;
    for (int64_t u = wk.u0, i = 0; u < wk.u1; ++u, ++i) {
      const int st = (int)(i & 1);
      // one thread waits for the stage; the named barrier makes the decision uniform
      if (i >= NSTAGE) {
        if (pt == 0 && !tc::mbar_wait(&bar_empty[st], ph_empty[st], WAIT_TRIES)) s_abort = 1;
        ph_empty[st] ^= 1u;
      }
      tc::named_sync(1, NPROD);
      if (s_abort) break;
      const int64_t tile = wk.tile(u);
      if (tile != cur_tile) {
        tc::named_sync(1, NPROD);
        if (pt < TM) {
          const int64_t p = tile * TM + pt;
          sEp[pt] = p < a.P ? a.xE[p] : 0;
        }
        tc::named_sync(1, NPROD);
        cur_tile = tile;
      }
      uint8_t* sA = sm + st * STAGE;
      uint8_t* sY = sA + S * A_PLANE;
      const uint8_t* ysrc = a.img + (u % a.kwins) * (int64_t)(S * Y_PLANE);
      for (int q = pt; q < S * Y_PLANE / 16; q += NPROD) tc::cp_async16(sY + 16 * q, ysrc + 16 * q);
      slice_window<TRANS>(a, tile, u % a.kwins, sA, sEp, pt);
      tc::cp_async_wait_all();
      tc::fence_async_smem();
      tc::mbar_arrive(&bar_full[st]);
    }
  } else if (warp == 12) {
    // ---------------------------------------------------------- MMA issuer
    uint32_t ph_full[NSTAGE] = {0, 0}, ph_accempty = 0;
    const uint32_t idesc = tc::idesc_bf16_f32(TM, NN);
    for (int64_t u = wk.u0, i = 0; u < wk.u1; ++u, ++i) {
      const int st = (int)(i & 1);
      bool ok = true;
      if (lane == 0) {
        ok = tc::mbar_wait(&bar_full[st], ph_full[st], WAIT_TRIES);
        if (ok && i > 0) ok = tc::mbar_wait(&bar_accempty, ph_accempty, WAIT_TRIES);
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      ph_full[st] ^= 1u;
      if (i > 0) ph_accempty ^= 1u;
      if (!ok) s_abort = 1;
      if (s_abort) break;
      tc::fence_after_sync();
      if (lane == 0) {
        const bool fresh = wk.seg_first(u);
        const uint32_t a0 = tc::smem_addr(sm + st * STAGE);
        const uint32_t y0 = a0 + S * A_PLANE;
#pragma unroll 1
        for (int sa = 0; sa < S; ++sa)
#pragma unroll 1
          for (int sy = 0; sy < S - sa; ++sy) {
            const int w = sa + sy;
            const uint32_t col = w < EXACT_GROUPS ? 64u * w : COL_G5;
            // exact groups restart every window; the weight >= 5 sum once per segment
            const bool first = (sa == 0) && (w < EXACT_GROUPS || (w == EXACT_GROUPS && fresh));
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
              tc::mma_bf16(tmem + col, tc::desc_k_none(a0 + sa * A_PLANE + 256 * kk, LBO, SBO),
                           tc::desc_k_none(y0 + sy * Y_PLANE + 256 * kk, LBO, SBO), idesc,
                           (first && kk == 0) ? 0u : 1u);
          }
        tc::mma_commit(&bar_empty[st]);
        tc::mma_commit(&bar_accfull);
      }
      __syncwarp();
    }
  } else if (warp < 4) {
    // ---------------------------------------------------------- flush + epilogue
    uint32_t ph_accfull = 0;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
    for (int64_t u = wk.u0; u < wk.u1; ++u) {
      // lane 0 waits; the warp follows its decision (tcgen05.ld is warp-collective)
      bool ok = true;
      if (lane == 0) ok = tc::mbar_wait(&bar_accfull, ph_accfull, WAIT_TRIES);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      ph_accfull ^= 1u;
      if (!ok) s_abort = 1;
      if (!ok) break;
      tc::fence_after_sync();
      const bool fresh = wk.seg_first(u);
#pragma unroll 1
      for (int c0 = 0; c0 < NN; c0 += 16) {
        uint32_t g0[16], g1[16], g2[16], g3[16], g4[16], lo[16], hi[16];
        tc::tmem_ld16(trow + 0u + c0, g0);
        tc::tmem_ld16(trow + 64u + c0, g1);
        tc::tmem_ld16(trow + 128u + c0, g2);
        tc::tmem_ld16(trow + 192u + c0, g3);
        tc::tmem_ld16(trow + 256u + c0, g4);
        if (!fresh) {
          tc::tmem_ld16(trow + COL_ACC_LO + c0, lo);
          tc::tmem_ld16(trow + COL_ACC_HI + c0, hi);
        }
        tc::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n0 = exact_int(g0[i], 1.0f);
          const int n1 = exact_int(g1[i], 0x1p7f);
          const int n2 = exact_int(g2[i], 0x1p14f);
          const int n3 = exact_int(g3[i], 0x1p21f);
          const int n4 = exact_int(g4[i], 0x1p28f);
          const int64_t add = ((int64_t)n0 << 28) + ((int64_t)(n1 * 128 + n2) << 14) +
                              (int64_t)(n3 * 128 + n4);
          int64_t acc = fresh ? 0 : (int64_t)(((uint64_t)hi[i] << 32) | (uint64_t)lo[i]);
          acc += add;
          lo[i] = (uint32_t)((uint64_t)acc & 0xFFFFFFFFull);
          hi[i] = (uint32_t)((uint64_t)acc >> 32);
        }
        tmem_st16(trow + COL_ACC_LO + c0, lo);
        tmem_st16(trow + COL_ACC_HI + c0, hi);
      }
      tmem_st_wait();
      if (wk.seg_last(u)) {
        const int64_t tile = wk.tile(u);
        const bool full = (u - (a.kwins - 1) == tile * a.kwins) && (u - (a.kwins - 1) >= wk.u0);
        const int pl = 32 * warp + lane;
        const int64_t p = tile * TM + pl;
        const int ep = p < a.P ? a.xE[p] : 0;
        const int slot = (tile == first_tile) ? 0 : 1;
        double* wrow = a.part + ((cta * 2 + slot) * TM + pl) * NN;
#pragma unroll 1
        for (int c0 = 0; c0 < NN; c0 += 16) {
          uint32_t lo[16], hi[16], g5[16];
          tc::tmem_ld16(trow + COL_ACC_LO + c0, lo);
          tc::tmem_ld16(trow + COL_ACC_HI + c0, hi);
          tc::tmem_ld16(trow + COL_G5 + c0, g5);
          tc::tmem_ld_wait();
          if (p < a.P) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int c = c0 + i;
              if (c < a.N) {
                const int64_t acc = (int64_t)(((uint64_t)hi[i] << 32) | (uint64_t)lo[i]);
                const double sum = fma(__ll2double_rn(acc), 0x1p-28, (double)__uint_as_float(g5[i]));
                const double v = ldexp(sum, ep + syE[c] - EXP_OFFSET);
                if (full) {
                  double* dst = a.C + p * a.csp + (int64_t)c * a.csc;
                  *dst = (a.beta == 0.0) ? a.alpha * v : a.alpha * v + a.beta * (*dst);
                } else {
                  wrow[c] = v;
                }
              }
            }
          }
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&bar_accempty);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (s_abort && tid == 0) atomicOr(a.flags, FLAG_TIMEOUT);
  if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

// Combine the partial tiles of tiles split across CTAs, in CTA order.  Grid:
// (tiles, FIX_SPLIT); each CTA handles TM*NN/FIX_SPLIT elements of its tile.
constexpr int FIX_SPLIT = 32;

__global__ void __launch_bounds__(256) k_oz_fixup(OzArgs a, int G) {
  const int64_t t = blockIdx.x;
  const int64_t T = a.tiles * a.kwins;
  auto owner = [&](int64_t u) {
    int64_t c = u * G / T;
    while (c + 1 < G && (c + 1) * T / G <= u) ++c;
    while (c > 0 && c * T / G > u) --c;
    return c;
  };
  const int64_t cf = owner(t * a.kwins), cl = owner((t + 1) * a.kwins - 1);
  if (cf == cl) return;
  constexpr int PER = TM * NN / FIX_SPLIT;
  for (int e = blockIdx.y * PER + threadIdx.x; e < (int)(blockIdx.y + 1) * PER; e += 256) {
    const int r = e / NN, c = e % NN;
    const int64_t p = t * TM + r;
    if (p >= a.P || c >= a.N) continue;
    double s = 0.0;
    for (int64_t q = cf; q <= cl; ++q) {
      const int64_t q0 = q * T / G, q1 = (q + 1) * T / G;
      if (q0 >= q1) continue;  // a CTA with an empty range wrote nothing
      const int slot = (t == q0 / a.kwins) ? 0 : 1;
      s += a.part[((q * 2 + slot) * TM + r) * NN + c];
    }
    double* dst = a.C + p * a.csp + (int64_t)c * a.csc;
    *dst = (a.beta == 0.0) ? a.alpha * s : a.alpha * s + a.beta * (*dst);
  }
}

cudaError_t oz_rowcol_exponents(const double* X, int64_t ld, int64_t rows, int64_t cols,
                                int* rowE, int* colE, cudaStream_t st, bool accumulate_rows) {
  if (colE) {
    k_oz_colmaxexp<<<(unsigned)cols, 256, 0, st>>>(X, ld, rows, colE);
    cudaError_t e = launched();
    if (e != cudaSuccess) return e;
  }
  if (rowE) {
    if (!accumulate_rows) {
      cudaError_t e = cudaMemsetAsync(rowE, 0, rows * sizeof(int), st);
      if (e != cudaSuccess) return e;
    }
    const int64_t csplit = cols >= 256 ? 16 : 1;
    const int64_t cchunk = (cols + csplit - 1) / csplit;
    dim3 grid((unsigned)((rows + 255) / 256), (unsigned)((cols + cchunk - 1) / cchunk));
    k_oz_rowmaxexp<<<grid, 256, 0, st>>>(X, ld, rows, cols, cchunk, rowE);
    return launched();
  }
  return cudaSuccess;
}

cudaError_t ozgemm(bool trans, int64_t P, int64_t N, int64_t K, double alpha, const double* X,
                   int64_t ldx, const int* xE, const double* Y, int64_t ldy, double beta, GemmOut out,
                   const OzWorkspace& w, int* flags, cudaStream_t st) {
  if (P <= 0 || N <= 0) return cudaSuccess;
  if (N > NN || K <= 0) return cudaErrorInvalidValue;
  const int64_t kwins = (K + KW - 1) / KW;
  if (oz_img_bytes(K) > w.img_bytes) return cudaErrorInvalidValue;
  static bool attr_set[2] = {false, false};
  if (!attr_set[trans ? 1 : 0]) {
    cudaError_t e = cudaFuncSetAttribute(trans ? (const void*)k_ozgemm<true> : (const void*)k_ozgemm<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_DYN);
    if (e != cudaSuccess) return e;
    attr_set[trans ? 1 : 0] = true;
  }
  k_oz_colmaxexp<<<(unsigned)N, 256, 0, st>>>(Y, ldy, K, w.yE);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  const int64_t ythreads = kwins * NN * 4;
  k_oz_yslice<<<(unsigned)((ythreads + 255) / 256), 256, 0, st>>>(Y, ldy, K, (int)N, w.yE, w.img,
                                                                  kwins);
  e = launched();
  if (e != cudaSuccess) return e;
  OzArgs a;
  a.P = P;
  a.K = K;
  a.N = N;
  a.X = X;
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
  a.kwins = kwins;
  a.flags = flags;
  a.vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (ldx % 2 == 0);
  const int G = w.ctas;
  if (trans)
    k_ozgemm<true><<<G, NT, SMEM_DYN, st>>>(a);
  else
    k_ozgemm<false><<<G, NT, SMEM_DYN, st>>>(a);
  e = launched();
  if (e != cudaSuccess) return e;
  k_oz_fixup<<<dim3((unsigned)a.tiles, FIX_SPLIT), 256, 0, st>>>(a, G);
  return launched();
}

}  // namespace lra
