// Sparse sketch Y = X Omega (Alg. 1 step "A G_j" with a sparse Omega_j; Alg. 2
// steps 5-7, A B_j - z).  Each output column g gathers counts[g] columns of the
// column-major X.  HBM-bound: a thread owns two consecutive rows and issues one
// 16-byte load per gathered column (unrolled by 4 so several loads are in
// flight); consecutive threads read consecutive 16-byte words of the same
// column, so every warp touches whole 128-byte lines.  Duplicated column
// indices across output columns of a block hit in L2.
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

cudaError_t gather_sketch(const double* X, int64_t ldx, int64_t rows_x, const int* counts,
                          const int* rows, const double* vals, int cap, int64_t ncols, double* Y,
                          int64_t ldy, const double* shift, cudaStream_t st) {
  if (ncols <= 0 || rows_x <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t chunks = (rows_x + 2 * threads - 1) / (2 * threads);
  dim3 grid((unsigned)chunks, (unsigned)(ncols < 65535 ? ncols : 65535));
  const bool vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (ldx % 2 == 0);
  if (vec)
    k_gather<true><<<grid, threads, 0, st>>>(X, ldx, rows_x, counts, rows, vals, cap, ncols, Y,
                                             ldy, shift);
  else
    k_gather<false><<<grid, threads, 0, st>>>(X, ldx, rows_x, counts, rows, vals, cap, ncols, Y,
                                              ldy, shift);
  return launched();
}

}  // namespace lra
