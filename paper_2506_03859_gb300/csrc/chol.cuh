// The b x b Cholesky factor with its inverse (orth.cu's k_chol_inv and the fused
// Gram fixup + Cholesky of ozgemm.cu): one CTA of CHOL_NT threads.
#pragma once

#include <math.h>

#include "internal.cuh"

namespace lra {

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
// Closer still (every entry of S - I within 2^-40), X R^{-1} = X + X (R^{-1} - I)
// may take the correction term in FP32 (k_rinv_near_identity in orth.cu): the
// entries of R^{-1} - I = -Phi(S - I) are then within 2^-40, so FP32's relative
// error of (b + 4) 2^-24 in that term, which is at most 2^-40 sqrt(b) times X's
// row norm, stays below 2^-55 of that norm.  *near (when given) records the test.
constexpr double CHOL_NEAR_I_FP32 = 0x1p-40;

//
// Skip mode (dead != NULL, the first pass over a power-step panel): a failed
// pivot marks column c dependent instead of ending the factorisation.  Its
// reciprocal pivot is taken as 0, so row c of R beyond the diagonal and row c of
// Z are zero: the column updates nothing after it, no other column of R^{-1}
// refers to it, and column c of R^{-1} is zero (the caller replaces that column
// of X R^{-1}).
// The whole factorisation by one CTA of CHOL_NT threads (k_chol_inv, and the last
// CTA of the Gram's fixup in ozgemm.cu).  S is read once, with loads that bypass
// L1 (it may have been written by other CTAs of the same launch).
__device__ __forceinline__ void chol_inv_cta(const double* __restrict__ S, int b, double tau,
                                             double* __restrict__ Rinv, int* __restrict__ flags,
                                             int* __restrict__ dead, int* __restrict__ near) {
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
  int far = 0;   // an entry of S - I above 2^-34, or not finite
  int wide = 0;  // an entry of S - I above 2^-40, or not finite
  for (int e = t; e < b * b; e += CHOL_NT) {
    const int i = e % b, j = e / b;
    const double v = __ldcg(S + i + j * b);
    M[i][j] = v;
    Z[i][j] = (i == j) ? 1.0 : 0.0;
    const double dev = fabs(i == j ? v - 1.0 : v);
    far |= !(dev <= CHOL_NEAR_I);
    wide |= !(dev <= CHOL_NEAR_I_FP32);
  }
  const int any_wide = __syncthreads_or(wide);
  if (near && t == 0) *near = !any_wide;
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
  if (t < b) Sd[t] = __ldcg(S + t + t * b);
  if (t == 0) {
    const double d = __ldcg(S);
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


}  // namespace lra
