// Philox4x32-10 on the device, from its definition in J. K. Salmon et al.,
// "Parallel random numbers: as easy as 1, 2, 3" (SC'11), Sec. 3: per round two
// 32x32->64-bit products of counter words with fixed multipliers, the halves
// crossed with the other words and the key, the key advanced by a Weyl step.
//
// Stream conventions of this library (Omega_j for block j, column c, draw or
// row x; key = (seed_lo, seed_hi); counter = (x, j, c, tag)):
//  - fixed-zeta sparse sign: row = (u0 * n) >> 32, sign from bit 0 of u1;
//  - Bernoulli mask: u0 < floor(p 2^32); i.i.d. sparse sign sign = bit 0 of u1;
//  - Gaussian: Box-Muller on a = (k(u0,u1)+1) 2^-53 in (0,1] and
//    c = k(u2,u3) 2^-53 in [0,1), k(x,y) = (x >> 5) 2^26 + (y >> 6).
#pragma once

#include <stdint.h>

namespace lra {

struct U32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return U32x4{c0, c1, c2, c3};
}

// Standard normal value for (row r, block j, column c).
__device__ __forceinline__ double philox_gaussian(uint32_t r, uint32_t j, uint32_t c, uint32_t k0,
                                                  uint32_t k1, uint32_t tag) {
  const U32x4 u = philox4x32_10(r, j, c, tag, k0, k1);
  const uint64_t ka = ((uint64_t)(u.x >> 5) << 26) | (uint64_t)(u.y >> 6);
  const uint64_t kc = ((uint64_t)(u.z >> 5) << 26) | (uint64_t)(u.w >> 6);
  const double a = ((double)ka + 1.0) * 0x1p-53;
  const double cc = (double)kc * 0x1p-53;
  return sqrt(-2.0 * log(a)) * cospi(2.0 * cc);
}

}  // namespace lra
