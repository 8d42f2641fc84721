// Test matrices Omega_j on the device (arxiv 2506.03859 Sec. 2.2, Def. 2.1-2.4
// and the fixed-nonzeros sparse sign variant described after Def. 2.2).
// Every entry is a pure function of (seed, j, c, row or draw): resuming at
// block j, or sketching blocks in any order, reproduces Omega_j bit for bit.
#include "internal.cuh"
#include "philox.cuh"

namespace lra {

// One thread per column g of the nblk*b generated columns.  Draws rows until
// zeta distinct ones are accepted (rejecting repeats), at most 64*zeta+1024
// draws; stores them in acceptance order with value +-1/sqrt(zeta).
__global__ void k_omega_fixed_zeta(int64_t j0, int64_t ncols, int b, int64_t n, int zeta,
                                   double inv_scale, uint32_t k0, uint32_t k1, int cap,
                                   int* __restrict__ counts, int* __restrict__ rows,
                                   double* __restrict__ vals, int* __restrict__ flags) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ncols) return;
  const uint32_t j = (uint32_t)(j0 + g / b);
  const uint32_t c = (uint32_t)(g % b);
  int taken[LRA_MAX_ZETA];
  int cnt = 0;
  const int max_draws = 64 * zeta + 1024;
  for (int t = 0; t < max_draws && cnt < zeta; ++t) {
    const U32x4 u = philox4x32_10((uint32_t)t, j, c, TAG_SPARSE_SIGN, k0, k1);
    const int r = (int)(((uint64_t)u.x * (uint64_t)n) >> 32);
    bool dup = false;
    for (int q = 0; q < cnt; ++q) dup |= (taken[q] == r);
    if (dup) continue;
    taken[cnt] = r;
    rows[g * cap + cnt] = r;
    vals[g * cap + cnt] = (u.y & 1u) ? -inv_scale : inv_scale;
    ++cnt;
  }
  if (cnt < zeta) atomicOr(flags, FLAG_OMEGA_CAP);
  counts[g] = cnt;
}

__device__ __forceinline__ double mask_value(int kind, bool on, const U32x4& u, uint32_t r,
                                             uint32_t j, uint32_t c, double inv_scale, uint32_t k0,
                                             uint32_t k1) {
  if (!on) return 0.0;
  switch (kind) {
    case LRA_OMEGA_SPARSE_SIGN_IID:
      return (u.y & 1u) ? -inv_scale : inv_scale;
    case LRA_OMEGA_SPARSE_GAUSSIAN:
      return philox_gaussian(r, j, c, k0, k1, TAG_GAUSS) * inv_scale;
    default:  // Bernoulli and standardized Bernoulli: the Bernoulli entry itself
      return 1.0;
  }
}

// One CTA (256 threads) per column: rows in increasing order, compacted with a
// block-wide prefix count so the output order is deterministic.
__global__ void __launch_bounds__(256) k_omega_mask(int64_t j0, int b, int64_t n, int kind,
                                                    uint64_t thr, double inv_scale, uint32_t k0,
                                                    uint32_t k1, int cap, int* __restrict__ counts,
                                                    int* __restrict__ rows,
                                                    double* __restrict__ vals) {
  __shared__ int warp_tot[8];
  __shared__ int s_base;
  const int64_t g = blockIdx.x;
  const uint32_t j = (uint32_t)(j0 + g / b);
  const uint32_t c = (uint32_t)(g % b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += 256) {
    const int64_t r = base + threadIdx.x;
    bool on = false;
    double v = 0.0;
    if (r < n) {
      const U32x4 u = philox4x32_10((uint32_t)r, j, c, TAG_MASK, k0, k1);
      on = (uint64_t)u.x < thr;
      v = mask_value(kind, on, u, (uint32_t)r, j, c, inv_scale, k0, k1);
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, on);
    const int before = __popc(ballot & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[wid] = __popc(ballot);
    __syncthreads();
    int off = s_base;
    for (int q = 0; q < wid; ++q) off += warp_tot[q];
    if (on) {
      rows[g * cap + off + before] = (int)r;
      vals[g * cap + off + before] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int q = 0; q < 8; ++q) t += warp_tot[q];
      s_base += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[g] = s_base;
}

__global__ void k_omega_dense(int64_t j0, int64_t ncols, int b, int64_t n, int kind, uint64_t thr,
                              double p, double inv_scale, uint32_t k0, uint32_t k1,
                              double* __restrict__ Om, int64_t ldo) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t g = blockIdx.y;
  if (r >= n || g >= ncols) return;
  const uint32_t j = (uint32_t)(j0 + g / b);
  const uint32_t c = (uint32_t)(g % b);
  double v;
  if (kind == LRA_OMEGA_GAUSSIAN) {
    v = philox_gaussian((uint32_t)r, j, c, k0, k1, TAG_GAUSS);
  } else {
    const U32x4 u = philox4x32_10((uint32_t)r, j, c, TAG_MASK, k0, k1);
    const bool on = (uint64_t)u.x < thr;
    if (kind == LRA_OMEGA_STD_BERNOULLI)
      v = on ? 1.0 - p : -p;  // B_j - p 1 1^T: Alg. 2's A B_j - z with the scale dropped
    else
      v = mask_value(kind, on, u, (uint32_t)r, j, c, inv_scale, k0, k1);
  }
  Om[r + g * ldo] = v;
}

cudaError_t omega_sparse(const OmegaSpec& s, int64_t j0, int64_t nblk, int cap, int* counts,
                         int* rows, double* vals, int* flags, cudaStream_t st) {
  const int64_t ncols = nblk * s.b;
  if (ncols <= 0) return cudaSuccess;
  if (s.kind == LRA_OMEGA_SPARSE_SIGN) {
    const int threads = 128;
    k_omega_fixed_zeta<<<(unsigned)((ncols + threads - 1) / threads), threads, 0, st>>>(
        j0, ncols, s.b, s.n, s.zeta, s.inv_scale, s.k0, s.k1, cap, counts, rows, vals, flags);
    return launched();
  }
  k_omega_mask<<<(unsigned)ncols, 256, 0, st>>>(j0, s.b, s.n, s.kind, s.thr, s.inv_scale, s.k0,
                                                s.k1, cap, counts, rows, vals);
  return launched();
}

__global__ void __launch_bounds__(256) k_fill_dead(double* __restrict__ X, int64_t ldx, int64_t rows,
                                                   const int* __restrict__ dead, uint32_t k0,
                                                   uint32_t k1, uint32_t j, uint32_t c0) {
  const int c = blockIdx.y;
  if (!dead[c]) return;
  const int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (r >= rows) return;
  const U32x4 u = philox4x32_10((uint32_t)r, j, c0 + (uint32_t)c, TAG_FILL, k0, k1);
  const double v = 1.0 / sqrt((double)rows);  // IEEE square root and division
  X[r + (int64_t)c * ldx] = (u.x & 1u) ? -v : v;
}

cudaError_t fill_dead(double* X, int64_t ldx, int64_t rows, int b, const int* dead, uint32_t k0,
                      uint32_t k1, int64_t j, int step, cudaStream_t st) {
  if (rows <= 0 || b <= 0) return cudaSuccess;
  dim3 grid((unsigned)((rows + 255) / 256), (unsigned)b);
  k_fill_dead<<<grid, 256, 0, st>>>(X, ldx, rows, dead, k0, k1, (uint32_t)j, (uint32_t)(64 * step));
  return launched();
}

cudaError_t omega_dense(const OmegaSpec& s, int64_t j0, int64_t nblk, double* Om, int64_t ldo,
                        cudaStream_t st) {
  const int64_t ncols = nblk * s.b;
  if (ncols <= 0) return cudaSuccess;
  dim3 grid((unsigned)((s.n + 255) / 256), (unsigned)ncols);
  k_omega_dense<<<grid, 256, 0, st>>>(j0, ncols, s.b, s.n, s.kind, s.thr, s.p, s.inv_scale, s.k0,
                                      s.k1, Om, ldo);
  return launched();
}

}  // namespace lra
