// Sparse sketch Y = X Omega (Alg. 1 step "A G_j" with a sparse Omega_j; Alg. 2
// steps 5-7, A B_j - z).  Each output column g gathers counts[g] columns of the
// column-major X.  A thread owns two consecutive rows and issues one 16-byte
// load per gathered column, all of a column's loads before any arithmetic;
// consecutive threads read consecutive 16-byte words of the same column, so
// every warp touches whole 128-byte lines.  Duplicated column indices across
// output columns of a block hit in L2.
#include "internal.cuh"

namespace lra {

template <bool VEC2>
__global__ void __launch_bounds__(256)
    k_gather(const double* __restrict__ X, int64_t ldx, int64_t rows_x,
             const int* __restrict__ counts, const int* __restrict__ rows,
             const double* __restrict__ vals, int cap, int64_t ncols, double* __restrict__ Y,
             int64_t ldy, const double* __restrict__ shift) {
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (i0 >= rows_x) return;
  const bool two = (i0 + 1) < rows_x;
  for (int64_t g = blockIdx.y; g < ncols; g += gridDim.y) {
    const int cnt = __ldg(counts + g);
    const int* rg = rows + g * cap;
    const double* vg = vals + g * cap;
    double acc0 = 0.0, acc1 = 0.0;
    int t = 0;
    if (VEC2 && two) {
      for (; t + 4 <= cnt; t += 4) {
        const int r0 = __ldg(rg + t), r1 = __ldg(rg + t + 1), r2 = __ldg(rg + t + 2),
                  r3 = __ldg(rg + t + 3);
        const double2 a0 = __ldg(reinterpret_cast<const double2*>(X + (int64_t)r0 * ldx + i0));
        const double2 a1 = __ldg(reinterpret_cast<const double2*>(X + (int64_t)r1 * ldx + i0));
        const double2 a2 = __ldg(reinterpret_cast<const double2*>(X + (int64_t)r2 * ldx + i0));
        const double2 a3 = __ldg(reinterpret_cast<const double2*>(X + (int64_t)r3 * ldx + i0));
        const double v0 = __ldg(vg + t), v1 = __ldg(vg + t + 1), v2 = __ldg(vg + t + 2),
                     v3 = __ldg(vg + t + 3);
        acc0 = fma(v0, a0.x, acc0);
        acc1 = fma(v0, a0.y, acc1);
        acc0 = fma(v1, a1.x, acc0);
        acc1 = fma(v1, a1.y, acc1);
        acc0 = fma(v2, a2.x, acc0);
        acc1 = fma(v2, a2.y, acc1);
        acc0 = fma(v3, a3.x, acc0);
        acc1 = fma(v3, a3.y, acc1);
      }
      for (; t < cnt; ++t) {
        const int r = __ldg(rg + t);
        const double2 a = __ldg(reinterpret_cast<const double2*>(X + (int64_t)r * ldx + i0));
        const double v = __ldg(vg + t);
        acc0 = fma(v, a.x, acc0);
        acc1 = fma(v, a.y, acc1);
      }
    } else {
      for (; t < cnt; ++t) {
        const int r = __ldg(rg + t);
        const double v = __ldg(vg + t);
        const double* col = X + (int64_t)r * ldx + i0;
        acc0 = fma(v, __ldg(col), acc0);
        if (two) acc1 = fma(v, __ldg(col + 1), acc1);
      }
    }
    if (shift) {
      acc0 -= __ldg(shift + i0);
      if (two) acc1 -= __ldg(shift + i0 + 1);
    }
    double* yg = Y + g * ldy + i0;
    yg[0] = acc0;
    if (two) yg[1] = acc1;
  }
}

// ---------------------------------------------------------------------------
// Omega entries of one magnitude (+-v: the sparse sign kinds; v = 1: the
// Bernoulli kinds).  On GB300 every FP64 add costs as much as a DFMA on a pipe
// delivering ~0.6 Tops/s, so summing zeta FP64 terms per output would bound
// the pass by the FP64 pipe, not by HBM.  Here the signed sum of the gathered
// doubles is taken exactly in 64-bit integer fixed point, aligned to the
// largest exponent among a row's terms (at most 16 terms: 5 bits of headroom),
// converted back to FP64 with round-to-nearest-even by integer operations, and
// multiplied by v once: one FP64 operation per output instead of zeta.
// The 53-bit significand M of a double (hi word h, lo word l), shifted to
// M * 2^(5 - d) for d = emax - E, as the 64-bit word (th:tl); d + 6 >= 64 (or a
// zero / subnormal input, which is given d = 127) yields 0.  Exact unless the
// term is more than 5 binades below the largest, then truncated below 2^-58 of it.
__device__ __forceinline__ void fixed_term32(uint32_t h, uint32_t l, int emax, uint32_t& th,
                                             uint32_t& tl) {
  const int E = (int)((h << 1) >> 21);
  const int k = (E != 0 ? emax - E : 127) + 6;     // right shift of M << 11
  const uint32_t mh = (h & 0x000FFFFFu) | 0x00100000u;
  const uint32_t vh = __funnelshift_l(l, mh, 11);  // (M << 11) is a 64-bit word
  const uint32_t vl = l << 11;
  if (k < 32) {
    tl = __funnelshift_r(vl, vh, k);
    th = vh >> k;
  } else {
    tl = k < 64 ? (vh >> (k - 32)) : 0u;
    th = 0u;
  }
}

// S * 2^(emax - 1080) * v: one int64 -> FP64 conversion and one multiply; the
// power of two goes into v's exponent field when that stays in the normal range.
__device__ __forceinline__ double pm_finish(int64_t S, int emax, double v) {
  if (emax == 2047) return __longlong_as_double(0x7FF8000000000000ll);  // Inf / NaN input
  if (emax == 0 || S == 0) return 0.0;
  const int64_t vb = __double_as_longlong(v);
  const int eb = (int)((vb >> 52) & 0x7FF) + emax - 1080;
  const double scale = (eb > 0 && eb < 2047) ? __longlong_as_double(vb + ((int64_t)(emax - 1080) << 52))
                                             : ldexp(v, emax - 1080);
  return __ll2double_rn(S) * scale;
}

template <bool VEC2, int MAXT>
__global__ void __launch_bounds__(256)
    k_gather_pm(const double* __restrict__ X, int64_t ldx, int64_t rows_x,
                const int* __restrict__ counts, const int* __restrict__ rows,
                const double* __restrict__ vals, int cap, int64_t ncols, double* __restrict__ Y,
                int64_t ldy, const double* __restrict__ shift, double v) {
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (i0 >= rows_x) return;
  const bool two = (i0 + 1) < rows_x;
  for (int64_t g = blockIdx.y; g < ncols; g += gridDim.y) {
    const int cnt = __ldg(counts + g);
    const int* rg = rows + g * cap;
    const double* vg = vals + g * cap;
    double y0, y1;
    if (cnt <= MAXT) {
      uint32_t h0[MAXT], l0[MAXT], h1[MAXT], l1[MAXT];
      bool neg[MAXT];
#pragma unroll
      for (int t = 0; t < MAXT; ++t) {
        h0[t] = l0[t] = h1[t] = l1[t] = 0u;
        neg[t] = false;
        if (t < cnt) {
          const double* col = X + (int64_t)__ldg(rg + t) * ldx + i0;
          neg[t] = __ldg(vg + t) < 0.0;
          double a0, a1 = 0.0;
          if (VEC2 && two) {
            const double2 q = __ldg(reinterpret_cast<const double2*>(col));
            a0 = q.x;
            a1 = q.y;
          } else {
            a0 = __ldg(col);
            if (two) a1 = __ldg(col + 1);
          }
          h0[t] = (uint32_t)__double2hiint(a0);
          l0[t] = (uint32_t)__double2loint(a0);
          h1[t] = (uint32_t)__double2hiint(a1);
          l1[t] = (uint32_t)__double2loint(a1);
        }
      }
      int e0 = 0, e1 = 0;
#pragma unroll
      for (int t = 0; t < MAXT; ++t) {
        e0 = max(e0, (int)((h0[t] << 1) >> 21));
        e1 = max(e1, (int)((h1[t] << 1) >> 21));
      }
      // signed sums: a term's sign is its own sign bit xor the Omega sign
      int64_t s0 = 0, s1 = 0;
#pragma unroll
      for (int t = 0; t < MAXT; ++t) {
        uint32_t th, tl;
        fixed_term32(h0[t], l0[t], e0, th, tl);
        const int64_t t0 = (int64_t)(((uint64_t)th << 32) | tl);
        s0 = (neg[t] != (bool)(h0[t] >> 31)) ? s0 - t0 : s0 + t0;
        fixed_term32(h1[t], l1[t], e1, th, tl);
        const int64_t t1 = (int64_t)(((uint64_t)th << 32) | tl);
        s1 = (neg[t] != (bool)(h1[t] >> 31)) ? s1 - t1 : s1 + t1;
      }
      // value = S * 2^(emax - 1080) * v
      y0 = pm_finish(s0, e0, v);
      y1 = pm_finish(s1, e1, v);
    } else {
      // long columns (large Bernoulli probability): FP64 multiply-adds
      y0 = 0.0;
      y1 = 0.0;
      for (int t = 0; t < cnt; ++t) {
        const double* col = X + (int64_t)__ldg(rg + t) * ldx + i0;
        const double w = __ldg(vg + t);
        y0 = fma(w, __ldg(col), y0);
        if (two) y1 = fma(w, __ldg(col + 1), y1);
      }
    }
    if (shift) {
      y0 -= __ldg(shift + i0);
      if (two) y1 -= __ldg(shift + i0 + 1);
    }
    double* yg = Y + g * ldy + i0;
    yg[0] = y0;
    if (two) yg[1] = y1;
  }
}

cudaError_t gather_sketch(const double* X, int64_t ldx, int64_t rows_x, const int* counts,
                          const int* rows, const double* vals, int cap, int64_t ncols, double* Y,
                          int64_t ldy, const double* shift, double pm_scale, cudaStream_t st) {
  if (ncols <= 0 || rows_x <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t chunks = (rows_x + 2 * threads - 1) / (2 * threads);
  dim3 grid((unsigned)chunks, (unsigned)(ncols < 65535 ? ncols : 65535));
  const bool vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (ldx % 2 == 0);
  if (pm_scale > 0.0) {
#define LRA_PM(V, T)                                                                            \
  k_gather_pm<V, T><<<grid, threads, 0, st>>>(X, ldx, rows_x, counts, rows, vals, cap, ncols, Y, \
                                              ldy, shift, pm_scale)
    if (cap <= 4) {
      if (vec) LRA_PM(true, 4); else LRA_PM(false, 4);
    } else if (cap <= 8) {
      if (vec) LRA_PM(true, 8); else LRA_PM(false, 8);
    } else {
      if (vec) LRA_PM(true, 16); else LRA_PM(false, 16);
    }
#undef LRA_PM
    return launched();
  }
  if (vec)
    k_gather<true><<<grid, threads, 0, st>>>(X, ldx, rows_x, counts, rows, vals, cap, ncols, Y,
                                             ldy, shift);
  else
    k_gather<false><<<grid, threads, 0, st>>>(X, ldx, rows_x, counts, rows, vals, cap, ncols, Y,
                                              ldy, shift);
  return launched();
}

}  // namespace lra
