// FP64-accurate skinny GEMM on the tcgen05 tensor cores: C = alpha op(X) Y + beta C
// with X, Y, C in FP64 and N <= 64.  These are the full passes over A of the
// farPCA block (arxiv 2506.03859 Alg. 1 steps A^T(A G_j), A G_j, A^T Y_j) and the
// smaller products of the projection and orthonormalisation steps.
//
// GB300's FP64 pipe delivers about 1.2 TFLOP/s, while such a pass streams A once
// from HBM: run as FP64 FMAs it is ~60x slower than the memory bound.  Instead
// every operand is cut, error-free, into bf16 slices (the splitting idea of
// Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 2012):
//
//   Scaling.  Row p of op(X) has largest biased exponent ex_p, column c of Y
//   ey_c.  x is turned into the signed integer N = trunc(x 2^(1077 - ex_p)),
//   |N| < 2^55, and written in base 256 with seven digits d_0..d_6 (d_0 the most
//   significant): N = sum_s d_s 256^(6-s), d_0 in [-128, 128], d_1..6 in
//   [-128, 127].  Every digit is an integer of at most 8 significant bits, exact
//   in bf16.  Y is cut the same way into digits e_0..e_6.
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
// pairs take 11 MMAs per 16 values of K (4 for w <= 3, 7 for w >= 4).
//
// Work split: one CTA per SM walks a contiguous range of (row tile, 32-deep
// stage) units ("stream-K"); tiles whose stages span two or more CTAs are
// written as partial sums and combined by a fixup kernel in a fixed order.
// Inside a CTA the work is pipelined by warp role: eight producer warps load a
// 128 x 32 block of op(X) one stage ahead into registers, cut it into the seven
// digit planes of a shared-memory stage (two stages, K-major core-matrix layout),
// while a bulk copy brings the pre-cut 64 x 32 block of Y; one thread issues
// the MMAs; four warps read the exact sums from TMEM at the end of each 64-deep
// window, re-arm them, and write the tile.  The MMAs of weight >= 4 of a window
// are issued before the wait for that re-arming, so the flush overlaps them.
// mbarriers hand stages and accumulators between the roles; every wait is bounded.
#include <math.h>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace lra {

namespace {
constexpr int S = 7;                     // digits per operand
constexpr int TM = 128;                  // rows of op(X) per tile
constexpr int KS = 32;                   // K per pipeline stage
constexpr int NN = 64;                   // output columns (N padded)
constexpr int NFLUSH = 128;              // flush threads (warps 0..3)
constexpr int NPROD = 256;               // producer threads (warps 4..11)
constexpr int MMA_WARP = 12;
constexpr int NT = NFLUSH + NPROD + 32;
constexpr int A_PLANE = TM * KS * 2;     // bytes of one digit plane of the op(X) block
constexpr int Y_PLANE = NN * KS * 2;     // bytes of one digit plane of the Y block
constexpr int Y_STAGE = S * Y_PLANE;     // the Y part of a stage (one bulk copy)
constexpr int STAGE = S * A_PLANE + Y_STAGE;
constexpr int NSTAGE = 2;
constexpr int SMEM_DYN = NSTAGE * STAGE + 1024;
constexpr uint32_t LBO = 128, SBO = 512;  // core-matrix strides (K, rows)
constexpr uint32_t TMEM_COLS = 512;       // weights 0..6: columns 0..447
constexpr uint32_t COL_ACC_LO = 448, COL_ACC_HI = 480;  // int64 sums of output columns 32..63
constexpr uint32_t MAGIC = 0x4B400000u;   // bits of 1.5 * 2^23
constexpr long WAIT_TRIES = 1L << 22;
constexpr int EXP_OFFSET = 2058;          // 2 * 1077 - 96: see the scaling above
constexpr int64_t MAX_K = int64_t(1) << 24;
}  // namespace

int64_t oz_img_bytes(int64_t K) { return (K + KS - 1) / KS * Y_STAGE; }
int64_t oz_part_elems(int ctas) { return (int64_t)ctas * 2 * TM * NN; }
int64_t oz_max_k() { return MAX_K; }

// Offset of element (row, k), k < 32, in the K-major core-matrix layout of a
// stage plane: core (row/8, k/8) at ((row/8)*4 + k/8)*128, row-major inside.
__host__ __device__ __forceinline__ uint32_t core_offset(uint32_t row, uint32_t k) {
  return (((row >> 3) << 2) + (k >> 3)) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

// N + BIAS as two 32-bit words, N = trunc(x 2^(1077 - emax)) (emax >= the
// biased exponent of x; zero and subnormal x give 0) and BIAS = 128 in each of
// the six low bytes: the bytes of N + BIAS, minus 128, are the base-256 digits
// of N below the top one, and its bits 48.. (signed) are the top digit.
__device__ __forceinline__ void biased_fixed(double x, int emax, uint32_t& nh, uint32_t& nl) {
  const uint32_t h = (uint32_t)__double2hiint(x), l = (uint32_t)__double2loint(x);
  const int E = (int)((h >> 20) & 0x7FFu);
  const uint32_t mh = (h & 0x000FFFFFu) | 0x00100000u;  // significand M = mh:l
  const uint32_t vh = __funnelshift_l(l, mh, 10);      // M << 10, high word
  const uint32_t vl = l << 10;
  const int k = (E != 0 ? emax - E : 64) + 8;          // |N| = (M << 10) >> k
  uint32_t rh, rl;
  if (k < 32) {
    rl = __funnelshift_r(vl, vh, k);
    rh = vh >> k;
  } else {
    rl = k < 64 ? vh >> (k - 32) : 0u;
    rh = 0u;
  }
  const uint32_t s = (uint32_t)((int)h >> 31);  // 0, or all ones for negative x
  uint64_t v = ((uint64_t)(rh ^ s) << 32) | (uint64_t)(rl ^ s);
  v += 0x0000808080808080ull + (uint64_t)(s & 1u);  // two's complement, plus BIAS
  nh = (uint32_t)(v >> 32);
  nl = (uint32_t)v;
}

// Digit SL (0 = most significant) of (nh, nl) as a float: the byte is dropped
// into the mantissa of 2^23 and 2^23 + 128 subtracted, exactly.
template <int SL>
__device__ __forceinline__ float digit_f(uint32_t nh, uint32_t nl) {
  if (SL == 0) return __int_as_float(0x4B000080 + ((int)nh >> 16)) - 8388736.0f;
  const uint32_t w = (SL <= 2) ? nh : nl;
  constexpr uint32_t byte = (SL <= 2) ? (2 - SL) : (6 - SL);
  return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7650u | byte)) - 8388736.0f;
}

// Two floats holding bf16-exact values -> packed bf16 pair (lo in the low half).
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632u);
}

// Eight consecutive K values of one row (or column) -> one 16-byte chunk in each
// of the seven digit planes at dst, dst + plane, ...
__device__ __forceinline__ void cut8(const double* v, int emax, uint8_t* dst, int plane) {
  uint32_t h[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) biased_fixed(v[i], emax, h[i], l[i]);
#define LRA_CUT(SL)                                                                   \
  {                                                                                   \
    uint4 q;                                                                          \
    q.x = pack_bf16(digit_f<SL>(h[0], l[0]), digit_f<SL>(h[1], l[1]));                \
    q.y = pack_bf16(digit_f<SL>(h[2], l[2]), digit_f<SL>(h[3], l[3]));                \
    q.z = pack_bf16(digit_f<SL>(h[4], l[4]), digit_f<SL>(h[5], l[5]));                \
    q.w = pack_bf16(digit_f<SL>(h[6], l[6]), digit_f<SL>(h[7], l[7]));                \
    *reinterpret_cast<uint4*>(dst + (SL) * plane) = q;                                \
  }
  LRA_CUT(0) LRA_CUT(1) LRA_CUT(2) LRA_CUT(3) LRA_CUT(4) LRA_CUT(5) LRA_CUT(6)
#undef LRA_CUT
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

// Pre-cut Y: stage u of the image holds the seven 64 x 32 (N x K) digit planes
// of K values 32u .. 32u + 31 in the core-matrix layout.  One thread per
// (stage, column c, 8-wide k chunk j).
__global__ void __launch_bounds__(256) k_oz_ycut(const double* __restrict__ Y, int64_t ldy,
                                                 int64_t K, int N, const int* __restrict__ yE,
                                                 uint8_t* __restrict__ img, int64_t kst) {
  const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (idx >= kst * NN * 4) return;
  const int j = (int)(idx & 3);
  const int c = (int)((idx >> 2) & (NN - 1));
  const int64_t u = idx >> 8;
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
  int64_t ldx;
  const int* xE;       // biased max exponent of each row of op(X)
  const int* yE;       // biased max exponent of each column of Y
  const uint8_t* img;  // pre-cut Y
  double alpha, beta;
  double* C;
  int64_t csp, csc;
  double* part;        // [cta][2][NN][TM] partial tiles
  int64_t tiles, kst;  // row tiles; 32-deep stages per tile
  int* flags;
  bool vec;            // 16-byte loads allowed (trans layout)
};

// The CTA's stages: a contiguous range [u0, u1) of (tile, stage) units,
// tile-major.  A segment is the part of the range inside one tile; a window is
// one or two consecutive stages of a segment, aligned to even stage indices.
struct Walk {
  int64_t u0, u1, kst;
  __device__ __forceinline__ int64_t tile(int64_t u) const { return u / kst; }
  __device__ __forceinline__ bool seg_first(int64_t u) const { return u == u0 || u % kst == 0; }
  __device__ __forceinline__ bool seg_last(int64_t u) const {
    return u + 1 == u1 || (u + 1) % kst == 0;
  }
  __device__ __forceinline__ bool win_first(int64_t u) const {
    return seg_first(u) || ((u % kst) & 1) == 0;
  }
  __device__ __forceinline__ bool win_last(int64_t u) const {
    return seg_last(u) || ((u % kst) & 1) == 1;
  }
};

// A producer thread's share of one stage: 16 values of op(X).  TRANS == false:
// op(X)[p, k] = X[p + k*ldx], the thread takes row 32 (pw % 4) + lane and 16
// consecutive k (coalesced across the warp).  TRANS == true: op(X)[p, k] =
// X[k + p*ldx]; each warp instruction covers one 8 x 8 core matrix, lane ->
// (row r8 = lane % 8, k pair lane / 8).
template <bool TRANS>
__device__ __forceinline__ void fetch(const OzArgs& a, int64_t u, int pw, int lane, double (&v)[16]) {
  const int64_t tile = u / a.kst, k0 = (u % a.kst) * KS;
  if (!TRANS) {
    const int64_t p = tile * TM + 32 * (pw & 3) + lane, kb = k0 + 16 * (pw >> 2);
    const bool in = p < a.P;
#pragma unroll
    for (int i = 0; i < 16; ++i)
      v[i] = (in && kb + i < a.K) ? __ldg(a.X + p + (kb + i) * a.ldx) : 0.0;
  } else {
    const int r8 = lane & 7, q = lane >> 3;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int core = pw + 8 * i, rg = core >> 2, kc = core & 3;
      const int64_t p = tile * TM + rg * 8 + r8, k = k0 + kc * 8 + 2 * q;
      v[2 * i] = 0.0;
      v[2 * i + 1] = 0.0;
      if (p < a.P) {
        const double* src = a.X + k + p * a.ldx;
        if (a.vec && k + 1 < a.K) {
          const double2 t = __ldg(reinterpret_cast<const double2*>(src));
          v[2 * i] = t.x;
          v[2 * i + 1] = t.y;
        } else {
          if (k < a.K) v[2 * i] = __ldg(src);
          if (k + 1 < a.K) v[2 * i + 1] = __ldg(src + 1);
        }
      }
    }
  }
}

// Cut the thread's 16 values into the stage; sE = row exponents of the tile.
template <bool TRANS>
__device__ __forceinline__ void cut_stage(const double (&v)[16], const int* sE, uint8_t* sA, int pw,
                                          int lane) {
  if (!TRANS) {
    const uint32_t row = 32 * (pw & 3) + lane, kb = 16 * (pw >> 2);
    const int e = sE[row];
    cut8(v, e, sA + core_offset(row, kb), A_PLANE);
    cut8(v + 8, e, sA + core_offset(row, kb + 8), A_PLANE);
  } else {
    const int r8 = lane & 7, q = lane >> 3;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int core = pw + 8 * i;
      const int e = sE[(core >> 2) * 8 + r8];
      uint8_t* dst = sA + core * 128 + r8 * 16 + q * 4;
      uint32_t h0, l0, h1, l1;
      biased_fixed(v[2 * i], e, h0, l0);
      biased_fixed(v[2 * i + 1], e, h1, l1);
#define LRA_CUT2(SL) \
  *reinterpret_cast<uint32_t*>(dst + (SL) * A_PLANE) = pack_bf16(digit_f<SL>(h0, l0), digit_f<SL>(h1, l1));
      LRA_CUT2(0) LRA_CUT2(1) LRA_CUT2(2) LRA_CUT2(3) LRA_CUT2(4) LRA_CUT2(5) LRA_CUT2(6)
#undef LRA_CUT2
    }
  }
}

// One MMA of X digit plane s against Y planes t0 .. t0+c-1 into the weight
// columns 64 (s + t0) .. ; kk selects the 16-deep half of the stage.
__device__ __forceinline__ void mma_group(uint32_t tmem, uint32_t a0, uint32_t y0, int s, int t0,
                                          int c, int kk, uint32_t accumulate) {
  const uint32_t idesc = tc::idesc_bf16_f32(TM, 64u * (uint32_t)c);
  tc::mma_bf16(tmem + 64u * (uint32_t)(s + t0),
               tc::desc_k_none(a0 + (uint32_t)s * A_PLANE + 256u * kk, LBO, SBO),
               tc::desc_k_none(y0 + (uint32_t)t0 * Y_PLANE + 256u * kk, LBO, SBO), idesc, accumulate);
}

template <bool TRANS>
__global__ void __launch_bounds__(NT, 1) k_ozgemm(OzArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_accfull, bar_accempty;
  __shared__ int syE[NN];
  __shared__ int sEx[2][TM];  // producers: row exponents of tiles (by tile parity)
  __shared__ volatile int s_abort;
  __shared__ volatile int s_pgo[2];  // producers: go on with iteration i (slot i % 2)
  const uint32_t raw = tc::smem_addr(smem_raw);
  uint8_t* sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t T = a.tiles * a.kst;
  const int64_t G = gridDim.x, cta = blockIdx.x;
  const Walk wk{cta * T / G, (cta + 1) * T / G, a.kst};
  if (wk.u0 >= wk.u1) return;

  if (warp == 0) tc::tmem_alloc(&s_tmem, TMEM_COLS);
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      tc::mbar_init(&bar_full[s], NPROD + 1);  // + the arrival that carries the Y bytes
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

  if (warp >= 4 && warp < MMA_WARP) {
    // ---------------------------------------------------------- producers
    const int pt = tid - NFLUSH, pw = pt >> 5;
    uint32_t ph_empty[NSTAGE] = {0, 0};
    // row exponents of a tile in sEx[tile % 2], written while the first stage of
    // the tile is fetched (one iteration ahead of its use, behind a named barrier)
    auto load_exps = [&](int64_t tile) {
      if (pt < TM) {
        const int64_t p = tile * TM + pt;
        sEx[tile & 1][pt] = p < a.P ? __ldg(a.xE + p) : 0;
      }
    };
    double v[16];
    load_exps(wk.tile(wk.u0));
    fetch<TRANS>(a, wk.u0, pw, lane, v);
    for (int64_t u = wk.u0, i = 0; u < wk.u1; ++u, ++i) {
      const int st = (int)(i & 1);
      // Thread 0 waits for the stage and decides whether to go on; the decision is
      // published in slot i % 2 before the named barrier and read after it, so all
      // producers leave the loop in the same iteration (slot i % 2 is next written
      // in iteration i + 2, after every producer has passed barrier i + 1).
      if (pt == 0) {
        bool go = s_abort == 0;
        if (go && i >= NSTAGE) go = tc::mbar_wait(&bar_empty[st], ph_empty[st], WAIT_TRIES);
        if (!go) s_abort = 1;
        s_pgo[i & 1] = go ? 1 : 0;
      }
      if (i >= NSTAGE) ph_empty[st] ^= 1u;
      tc::named_sync(1, NPROD);
      if (!s_pgo[i & 1]) break;
      uint8_t* sA = sm + st * STAGE;
      if (pt == 0) {
        tc::mbar_arrive_expect_tx(&bar_full[st], Y_STAGE);
        tc::bulk_g2s(sA + S * A_PLANE, a.img + (u % a.kst) * (int64_t)Y_STAGE, Y_STAGE,
                     &bar_full[st]);
      }
      // next stage's values are in flight while this one is cut
      double vn[16];
      if (u + 1 < wk.u1) {
        if (wk.tile(u + 1) != wk.tile(u)) load_exps(wk.tile(u + 1));
        fetch<TRANS>(a, u + 1, pw, lane, vn);
      }
      cut_stage<TRANS>(v, sEx[wk.tile(u) & 1], sA, pw, lane);
      tc::fence_async_smem();
      tc::mbar_arrive(&bar_full[st]);
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = vn[q];
    }
  } else if (warp == MMA_WARP) {
    // ---------------------------------------------------------- MMA issuer (one thread)
    if (lane == 0) {
      uint32_t ph_full[NSTAGE] = {0, 0}, ph_ae = 0;
      for (int64_t u = wk.u0, i = 0; u < wk.u1; ++u, ++i) {
        const int st = (int)(i & 1);
        if (!tc::mbar_wait(&bar_full[st], ph_full[st], WAIT_TRIES)) {
          s_abort = 1;
          break;
        }
        ph_full[st] ^= 1u;
        tc::fence_after_sync();
        const bool sf = wk.seg_first(u);
        // a new segment: the flush must have read the previous one's FP32 sums
        if (sf) {
          if (!tc::mbar_wait(&bar_accempty, ph_ae, WAIT_TRIES)) {
            s_abort = 1;
            break;
          }
          ph_ae ^= 1u;
          tc::fence_after_sync();
        }
        const uint32_t a0 = tc::smem_addr(sm + st * STAGE);
        const uint32_t y0 = a0 + S * A_PLANE;
        // weights 4..6 (FP32 over the segment); the first MMA of a segment starts them
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          mma_group(tmem, a0, y0, 0, 4, 3, kk, (sf && kk == 0) ? 0u : 1u);
          mma_group(tmem, a0, y0, 1, 3, 3, kk, 1u);
          mma_group(tmem, a0, y0, 2, 2, 3, kk, 1u);
          mma_group(tmem, a0, y0, 3, 1, 3, kk, 1u);
          mma_group(tmem, a0, y0, 4, 0, 3, kk, 1u);
          mma_group(tmem, a0, y0, 5, 0, 2, kk, 1u);
          mma_group(tmem, a0, y0, 6, 0, 1, kk, 1u);
        }
        // weights 0..3 (exact per window): wait until the flush has re-armed them
        if (wk.win_first(u) && !sf) {
          if (!tc::mbar_wait(&bar_accempty, ph_ae, WAIT_TRIES)) {
            s_abort = 1;
            break;
          }
          ph_ae ^= 1u;
          tc::fence_after_sync();
        }
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          mma_group(tmem, a0, y0, 0, 0, 4, kk, 1u);
          mma_group(tmem, a0, y0, 1, 0, 3, kk, 1u);
          mma_group(tmem, a0, y0, 2, 0, 2, kk, 1u);
          mma_group(tmem, a0, y0, 3, 0, 1, kk, 1u);
        }
        tc::mma_commit(&bar_empty[st]);
        if (wk.win_last(u)) tc::mma_commit(&bar_accfull);
      }
    }
    __syncwarp();
  } else if (warp < 4) {
    // ---------------------------------------------------------- flush + epilogue
    // warp w owns TMEM lanes / tile rows 32 w .. 32 w + 31 (one row per thread) and
    // all 64 output columns: the int64 sums of columns 0..31 live in registers,
    // those of columns 32..63 in TMEM columns COL_ACC_LO / COL_ACC_HI.
    const uint32_t tb = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
      for (int j = 0; j < 8; ++j) tc::tmem_st8_splat(tb + 64u * w + 8u * j, MAGIC);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      tc::tmem_st8_splat(tb + COL_ACC_LO + 8u * j, 0u);
      tc::tmem_st8_splat(tb + COL_ACC_HI + 8u * j, 0u);
    }
    tc::tmem_st_wait();
    tc::fence_before_sync();
    tc::mbar_arrive(&bar_accempty);

    int64_t acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0;
    uint32_t ph_af = 0;
    for (int64_t u = wk.u0; u < wk.u1; ++u) {
      if (!wk.win_last(u)) continue;
      // lane 0 waits; the warp follows its decision (tcgen05.ld is warp-collective)
      bool ok = true;
      if (lane == 0) ok = tc::mbar_wait(&bar_accfull, ph_af, WAIT_TRIES);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      ph_af ^= 1u;
      if (!ok) {
        s_abort = 1;
        break;
      }
      tc::fence_after_sync();
#pragma unroll
      for (int j = 0; j < 16; ++j) {  // 4 output columns at a time
        const uint32_t c4 = 4u * j;
        uint32_t g0[4], g1[4], g2[4], g3[4];
        tc::tmem_ld4(tb + c4, g0);
        tc::tmem_ld4(tb + 64u + c4, g1);
        tc::tmem_ld4(tb + 128u + c4, g2);
        tc::tmem_ld4(tb + 192u + c4, g3);
        tc::tmem_ld_wait();
        int64_t add[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          // (G_0 * 256 + G_1) and (G_2 * 256 + G_3), each exact in 32 bits
          const int hi = (int)(g0[i] * 256u + g1[i] - 257u * MAGIC);
          const int lo = (int)(g2[i] * 256u + g3[i] - 257u * MAGIC);
          add[i] = ((int64_t)hi << 16) + (int64_t)lo;
        }
        tc::tmem_st4_splat(tb + c4, MAGIC);
        tc::tmem_st4_splat(tb + 64u + c4, MAGIC);
        tc::tmem_st4_splat(tb + 128u + c4, MAGIC);
        tc::tmem_st4_splat(tb + 192u + c4, MAGIC);
        if (j < 8) {
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[4 * j + i] += add[i];
        } else {
          uint32_t lo[4], hi[4];
          tc::tmem_ld4(tb + COL_ACC_LO + c4 - 32u, lo);
          tc::tmem_ld4(tb + COL_ACC_HI + c4 - 32u, hi);
          tc::tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint64_t t = (((uint64_t)hi[i] << 32) | lo[i]) + (uint64_t)add[i];
            lo[i] = (uint32_t)t;
            hi[i] = (uint32_t)(t >> 32);
          }
          tc::tmem_st4(tb + COL_ACC_LO + c4 - 32u, lo);
          tc::tmem_st4(tb + COL_ACC_HI + c4 - 32u, hi);
        }
      }
      tc::tmem_st_wait();
      if (wk.seg_last(u)) {
        const int64_t tile = wk.tile(u);
        const bool full = (u + 1 - a.kst == tile * a.kst) && (tile * a.kst >= wk.u0);
        const int r = 32 * warp + lane;
        const int64_t p = tile * TM + r;
        const int ep = p < a.P ? __ldg(a.xE + p) : 0;
        const int slot = (tile == first_tile) ? 0 : 1;
        double* wp = a.part + (cta * 2 + slot) * (int64_t)(NN * TM) + r;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint32_t c4 = 4u * j;
          uint32_t g4[4], g5[4], g6[4], lo[4], hi[4];
          tc::tmem_ld4(tb + 256u + c4, g4);
          tc::tmem_ld4(tb + 320u + c4, g5);
          tc::tmem_ld4(tb + 384u + c4, g6);
          if (j >= 8) {
            tc::tmem_ld4(tb + COL_ACC_LO + c4 - 32u, lo);
            tc::tmem_ld4(tb + COL_ACC_HI + c4 - 32u, hi);
          }
          tc::tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int c = 4 * j + i;
            int64_t T;
            if (j < 8) {
              T = acc[c];
              acc[c] = 0;
            } else {
              T = (int64_t)(((uint64_t)hi[i] << 32) | lo[i]);
            }
            const double rest = (double)__uint_as_float(g4[i]) * 0x1p-32 +
                                (double)__uint_as_float(g5[i]) * 0x1p-40 +
                                (double)__uint_as_float(g6[i]) * 0x1p-48;
            const double sum = fma(__ll2double_rn(T), 0x1p-24, rest);
            if (p < a.P && c < a.N) {
              const double val = ldexp(sum, ep + syE[c] - EXP_OFFSET);
              if (full) {
                double* dst = a.C + p * a.csp + (int64_t)c * a.csc;
                *dst = (a.beta == 0.0) ? a.alpha * val : a.alpha * val + a.beta * (*dst);
              } else {
                wp[(int64_t)c * TM] = val;
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
  const int64_t T = a.tiles * a.kst;
  auto owner = [&](int64_t u) {
    int64_t c = u * G / T;
    while (c + 1 < G && (c + 1) * T / G <= u) ++c;
    while (c > 0 && c * T / G > u) --c;
    return c;
  };
  const int64_t cf = owner(t * a.kst), cl = owner((t + 1) * a.kst - 1);
  if (cf == cl) return;
  constexpr int PER = TM * NN / FIX_SPLIT;
  for (int e = blockIdx.y * PER + threadIdx.x; e < (int)(blockIdx.y + 1) * PER; e += 256) {
    const int r = e % TM, c = e / TM;
    const int64_t p = t * TM + r;
    if (p >= a.P || c >= a.N) continue;
    double s = 0.0;
    for (int64_t q = cf; q <= cl; ++q) {
      const int64_t q0 = q * T / G, q1 = (q + 1) * T / G;
      if (q0 >= q1) continue;  // a CTA with an empty range wrote nothing
      const int slot = (t == q0 / a.kst) ? 0 : 1;
      s += a.part[((q * 2 + slot) * NN + c) * TM + r];
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
  if (N > NN || K <= 0 || K > MAX_K) return cudaErrorInvalidValue;
  const int64_t kst = (K + KS - 1) / KS;
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
  const int64_t ythreads = kst * NN * 4;
  k_oz_ycut<<<(unsigned)((ythreads + 255) / 256), 256, 0, st>>>(Y, ldy, K, (int)N, w.yE, w.img, kst);
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
  a.kst = kst;
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
