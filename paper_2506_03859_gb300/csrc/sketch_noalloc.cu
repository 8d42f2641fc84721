// lra_sketch_noalloc: the sparse sketch Y = A [Omega_j0 ... Omega_{j0+nblk-1}]
// without any device allocation.
//
// Who needs it: callers that cannot allocate device memory once they are
// running -- a service that reserves its whole memory budget at start-up and
// forbids growth afterwards, or a host framework whose own allocator owns all
// device memory and would be bypassed (and possibly overrun) by a cudaMalloc,
// or latency-bound code that cannot afford the device synchronisation a
// cudaMalloc / cudaFree may cause.  lra_sketch needs a context, and
// lra_create allocates; this entry point needs none.
//
// The Omega structure (counts, row indices, values) that the generator writes
// and the gather kernel reads lives in one file-scope device array of
// LRA_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library keeps until
// the process exits.  Blocks are processed in chunks that fit the array.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace lra {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[LRA_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array in the current device's context.  In host
// code the array's name is only a host-side stand-in: the device address must
// come from cudaGetSymbolAddress.  It is looked up on every call (a cheap table
// lookup once the module is loaded), so an address is never reused across
// contexts: after cudaDeviceReset, or under another driver context on the same
// device, the module and its array may live elsewhere.  The first lookup in a
// context loads the library's device code there.
cudaError_t scratch_on_current_device(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

double noalloc_default_p(int kind, int64_t n, int zeta) {
  if (kind == LRA_OMEGA_SPARSE_GAUSSIAN && zeta > 0) return (double)zeta / (double)n;
  return fmax(1e-3, 10.0 / (double)n);
}

}  // namespace
}  // namespace lra

using namespace lra;

extern "C" lra_status lra_sketch_noalloc(const lra_matrix* A, const lra_params* params,
                                         int64_t j0, int64_t nblk, double* Y, int64_t ldy,
                                         void* cuda_stream) {
  if (!A || !A->data || !params || (nblk > 0 && !Y)) return LRA_ERR_INVALID_ARG;
  const int64_t m = A->m, n = A->n;
  const int b = params->b;
  if (m < 1 || n < 1 || m > INT32_MAX || n > INT32_MAX || A->lda < m || ldy < m)
    return LRA_ERR_INVALID_ARG;
  if (A->dtype != LRA_F64 && A->dtype != LRA_F32) return LRA_ERR_UNSUPPORTED;
  if (b < 1 || b > LRA_MAX_B || b > n) return LRA_ERR_INVALID_ARG;
  if (j0 < 0 || nblk < 0 || j0 + nblk > (int64_t)UINT32_MAX) return LRA_ERR_INVALID_ARG;
  if (!(params->p >= 0.0 && params->p < 1.0)) return LRA_ERR_INVALID_ARG;
  if (nblk == 0) return LRA_OK;

  // Omega of the kinds whose sketch is a pure gather (no rank-one shift, no dense pass)
  OmegaSpec os{};
  os.kind = params->kind;
  os.n = n;
  os.b = b;
  os.zeta = params->zeta;
  os.k0 = (uint32_t)(params->seed & 0xFFFFFFFFull);
  os.k1 = (uint32_t)(params->seed >> 32);
  os.inv_scale = 1.0;
  int cap = 0;
  switch (params->kind) {
    case LRA_OMEGA_SPARSE_SIGN:
      if (params->zeta < 1 || params->zeta > n || params->zeta > LRA_MAX_ZETA)
        return LRA_ERR_INVALID_ARG;
      os.inv_scale = 1.0 / sqrt((double)params->zeta);
      cap = params->zeta;
      break;
    case LRA_OMEGA_SPARSE_SIGN_IID:
    case LRA_OMEGA_SPARSE_GAUSSIAN:
    case LRA_OMEGA_BERNOULLI:
      if (params->zeta < 0) return LRA_ERR_INVALID_ARG;
      os.p = params->p > 0.0 ? params->p : noalloc_default_p(params->kind, n, params->zeta);
      os.thr = (uint64_t)floor(os.p * 4294967296.0);
      if (params->kind != LRA_OMEGA_BERNOULLI) os.inv_scale = 1.0 / sqrt(os.p);
      cap = (int)n;
      break;
    default:
      return LRA_ERR_UNSUPPORTED;  // Gaussian and standardized Bernoulli need a context
  }

  // Scratch layout: [flags int, padded to 256 B][counts int x cols][rows int x cols*cap][vals]
  const int64_t header = 256;
  const int64_t per_col = 4 + 12 * (int64_t)cap;
  const int64_t max_cols = (LRA_NOALLOC_SCRATCH_BYTES - header - 512) / per_col;
  if (max_cols < b) return LRA_ERR_INVALID_ARG;  // one block's Omega does not fit the array
  const int64_t chunk = std::min<int64_t>(max_cols / b, nblk);
  const int64_t cols = chunk * b;

  void* base = nullptr;
  cudaError_t e = scratch_on_current_device(&base);
  if (e != cudaSuccess) return LRA_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  uint8_t* sp = (uint8_t*)base;
  int* flags = (int*)sp;
  int* counts = (int*)(sp + header);
  int64_t off = header + ((cols * 4 + 255) / 256) * 256;
  int* rows = (int*)(sp + off);
  off += ((cols * (int64_t)cap * 4 + 255) / 256) * 256;
  double* vals = (double*)(sp + off);

  // the flag word must start at zero; the Omega arrays are fully rewritten per chunk
  if (cudaMemsetAsync(flags, 0, sizeof(int), st) != cudaSuccess) return LRA_ERR_CUDA;
  for (int64_t j = j0; j < j0 + nblk; j += chunk) {
    const int64_t nb = std::min(chunk, j0 + nblk - j);
    if (omega_sparse(os, j, nb, cap, counts, rows, vals, flags, st) != cudaSuccess)
      return LRA_ERR_CUDA;
    if (gather_sketch(A->data, A->dtype, A->lda, m, counts, rows, vals, cap, nb * b,
                      Y + (j - j0) * b * ldy, ldy,
                      nullptr, flags, st) != cudaSuccess)
      return LRA_ERR_CUDA;
  }
  int hflags = 0;
  if (cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return LRA_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LRA_ERR_CUDA;
  if (hflags & FLAG_OMEGA_CAP) return LRA_ERR_INVALID_ARG;
  if (hflags & FLAG_TIMEOUT) return LRA_ERR_TIMEOUT;
  return LRA_OK;
}
