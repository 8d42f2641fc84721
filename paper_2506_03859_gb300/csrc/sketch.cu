// Sparse sketch Y = X Omega (Alg. 1 step "A G_j" with a sparse Omega_j; Alg. 2
// steps 5-7, A B_j - z).  Each output column g gathers counts[g] columns of the
// column-major X, scaled by the Omega values, in FP64.  Duplicated column
// indices across output columns of a block hit in L2.
#include <algorithm>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace lra {

// ---------------------------------------------------------------------------
// The gathered column pieces are staged in shared memory by bulk copies: one CTA
// per (512-row chunk, output column); thread 0 copies up to 8 pieces of 4 KB per
// batch (completion counted on an mbarrier), then every thread reads its two rows
// of each piece with one 16-byte shared load and does the FP64 multiply-adds.
// One instruction moves a whole piece, so the load path carries no per-thread
// request queue, and at 32 KB of staging seven CTAs share an SM, which keeps
// enough bytes in flight for HBM.  A ragged last chunk, or an X whose columns are
// not 16-byte aligned, takes plain register loads.
constexpr int GR = 512;      // rows per CTA (two per thread)
constexpr int GBATCH = 8;    // pieces per batch
constexpr int GSMEM = GBATCH * GR * 8;  // 32 KB
constexpr long GWAIT_TRIES = 1L << 22;

// T: element type of X (double, or float converted exactly on load; the sums
// are FP64 either way).
template <typename T>
__global__ void __launch_bounds__(256) k_gather_staged(
    const T* __restrict__ X, int64_t ldx, int64_t rows_x, const int* __restrict__ counts,
    const int* __restrict__ rows, const double* __restrict__ vals, int cap, int64_t ncols,
    double* __restrict__ Y, int64_t ldy, const double* __restrict__ shift, bool aligned,
    int* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char sx_raw[];
  T* sx = reinterpret_cast<T*>(sx_raw);  // [GBATCH][GR]
  __shared__ __align__(8) uint64_t bar;
  const int64_t r0 = (int64_t)blockIdx.x * GR;
  const int nr = (int)((rows_x - r0) < GR ? (rows_x - r0) : GR);
  const bool staged = aligned && nr == GR;
  const int i = 2 * threadIdx.x;
  if (staged && threadIdx.x == 0) tc::mbar_init(&bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  for (int64_t g = blockIdx.y; g < ncols; g += gridDim.y) {
    const int cnt = __ldg(counts + g);
    const int* rg = rows + g * cap;
    const double* vg = vals + g * cap;
    double acc0 = 0.0, acc1 = 0.0;
    if (staged) {
      for (int t0 = 0; t0 < cnt; t0 += GBATCH) {
        const int nb = min(GBATCH, cnt - t0);
        if (threadIdx.x == 0) {
          int rr[GBATCH];
#pragma unroll
          for (int q = 0; q < GBATCH; ++q) rr[q] = q < nb ? __ldg(rg + t0 + q) : 0;
          tc::fence_async_smem();  // earlier reads of the buffer before the copies
          tc::mbar_arrive_expect_tx(&bar, (uint32_t)(nb * GR * sizeof(T)));
#pragma unroll
          for (int q = 0; q < GBATCH; ++q)
            if (q < nb)
              tc::bulk_g2s(sx + q * GR, X + (int64_t)rr[q] * ldx + r0, GR * sizeof(T), &bar);
        }
        double v[GBATCH];
#pragma unroll
        for (int q = 0; q < GBATCH; ++q) v[q] = q < nb ? __ldg(vg + t0 + q) : 0.0;
        const bool ok = tc::mbar_wait(&bar, phase, GWAIT_TRIES);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
          if (threadIdx.x == 0) {
            atomicOr(flags, FLAG_TIMEOUT);
            tc::mbar_wait(&bar, phase ^ 1u, GWAIT_TRIES);  // let copies in flight land
          }
          return;
        }
#pragma unroll
        for (int q = 0; q < GBATCH; ++q) {
          if (q < nb) {
            double a0, a1;
            if constexpr (sizeof(T) == 8) {
              const double2 a = reinterpret_cast<const double2*>(sx + q * GR)[threadIdx.x];
              a0 = a.x;
              a1 = a.y;
            } else {
              const float2 a = reinterpret_cast<const float2*>(sx + q * GR)[threadIdx.x];
              a0 = (double)a.x;
              a1 = (double)a.y;
            }
            acc0 = fma(v[q], a0, acc0);
            acc1 = fma(v[q], a1, acc1);
          }
        }
        __syncthreads();  // the buffer is refilled by the next batch
      }
    } else {
      for (int t = 0; t < cnt; ++t) {
        const T* col = X + (int64_t)__ldg(rg + t) * ldx + r0;
        const double v = __ldg(vg + t);
        if (i < nr) acc0 = fma(v, (double)__ldg(col + i), acc0);
        if (i + 1 < nr) acc1 = fma(v, (double)__ldg(col + i + 1), acc1);
      }
    }
    if (shift) {
      if (i < nr) acc0 -= __ldg(shift + r0 + i);
      if (i + 1 < nr) acc1 -= __ldg(shift + r0 + i + 1);
    }
    double* yg = Y + g * ldy + r0;
    if (i < nr) yg[i] = acc0;
    if (i + 1 < nr) yg[i + 1] = acc1;
  }
}

cudaError_t gather_prepare() {
  static std::atomic<bool> attr{false};  // concurrent first calls set it twice, harmlessly
  if (attr.load(std::memory_order_acquire)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute((const void*)k_gather_staged<double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, GSMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_gather_staged<float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, GSMEM);
  if (e == cudaSuccess) attr.store(true, std::memory_order_release);
  return e;
}

cudaError_t gather_sketch(const void* X, int dtype, int64_t ldx, int64_t rows_x, const int* counts,
                          const int* rows, const double* vals, int cap, int64_t ncols, double* Y,
                          int64_t ldy, const double* shift, int* flags, cudaStream_t st) {
  if (ncols <= 0 || rows_x <= 0) return cudaSuccess;
  cudaError_t e0 = gather_prepare();
  if (e0 != cudaSuccess) return e0;
  const int64_t chunks = (rows_x + GR - 1) / GR;
  dim3 grid((unsigned)chunks, (unsigned)std::min<int64_t>(ncols, 65535));
  // bulk copies start on 16-byte boundaries: the base, and every column start
  const int64_t esize = dtype == LRA_F32 ? 4 : 8;
  const bool aligned =
      ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && ((ldx * esize) % 16 == 0);
  if (dtype == LRA_F32)
    k_gather_staged<float><<<grid, 256, GSMEM, st>>>((const float*)X, ldx, rows_x, counts, rows,
                                                     vals, cap, ncols, Y, ldy, shift, aligned, flags);
  else
    k_gather_staged<double><<<grid, 256, GSMEM, st>>>((const double*)X, ldx, rows_x, counts, rows,
                                                      vals, cap, ncols, Y, ldy, shift, aligned,
                                                      flags);
  return launched();
}

}  // namespace lra
