// C ABI of the library (include/lra.h) and the host driver of the blocked
// farPCA loop (arxiv 2506.03859 Alg. 1, Alg. 2 for the standardized Bernoulli
// test matrix), written in its QB form (Sec. 2.1: farPCA equals randQB_EI plus
// a direct SVD for P = 0, 1, 2):
//
//   E = ||A||_F^2                                        (Alg. 1 step 1)
//   for j: Omega_j (Philox, device)                      (step 3 / Alg. 2 step 4)
//          S0 = A Omega_j  (Alg. 2: A B_j - z)            (steps 5-7)
//          P >= 1: W = A^T S0 - B^T (B Omega_j); G = orth(W);
//                  P-1 times W = A^T (A G) - B^T (B G), G = orth(W);  Y_j = A G
//                  (deflation W Z^{-1} W^T = B^T B, steps 5-6 / Alg. 2 steps 9-13)
//          P = 0:  Y_j = S0
//          Y' = (I - Q Q^T) Y_j twice; Q_j = orth(Y'); B_j = Q_j^T A  (step 9-10)
//          E -= ||B_j||_F^2; stop when E < eps^2 ||A||_F^2         (steps 10-11)
//
// orth(X) = X R^{-1} with R = chol(X^T X), applied twice (CholQR2): the Q factor
// of the QR factorisation with positive diag(R).  All device work is ordered on
// the context's stream; the host reads one small record per block (||B_j||_F^2
// and the error flags) for the stop test.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace lra {
std::atomic<uint64_t> g_launches{0};
}

using namespace lra;

namespace {

constexpr double PIVOT_TAU = 1e-13;
constexpr int64_t SPARSE_MAX_NNZ_PER_COL = 256;   // above this expected nnz, Omega is dense
constexpr int64_t SKETCH_SCRATCH_ENTRIES = 8 << 20;
constexpr int SVD_MAX_SWEEPS = 40;
constexpr double SVD_JACOBI_TOL = 1e-15;  // skip a pair when |c_pq| <= tol sqrt(|c_pp c_qq|)

struct Pinned {
  double v[4];
  int flags;
};

// The small pinned blocks through which every context reads its scalars back
// (one per context).  They come from page-locked chunks allocated once and
// kept for the process: releasing page-locked memory can synchronise the
// device, which would stall every other context at each destroy (the serving
// runtime creates and destroys contexts next to running ones).
class PinnedArena {
 public:
  Pinned* get() {
    std::lock_guard<std::mutex> lk(mu_);
    if (free_.empty()) {
      Pinned* chunk = nullptr;
      if (cudaMallocHost((void**)&chunk, sizeof(Pinned) * kChunk) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      for (int i = kChunk - 1; i >= 0; --i) free_.push_back(chunk + i);
    }
    Pinned* p = free_.back();
    free_.pop_back();
    return p;
  }
  void put(Pinned* p) {
    std::lock_guard<std::mutex> lk(mu_);
    free_.push_back(p);
  }

 private:
  static constexpr int kChunk = 256;
  std::mutex mu_;
  std::vector<Pinned*> free_;
};

PinnedArena& pinned_arena() {
  static PinnedArena* a = new PinnedArena();  // never destroyed: outlives every context
  return *a;
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct lra_ctx {
  int64_t m = 0, n = 0;
  lra_params prm{};
  cudaStream_t st = nullptr;
  int b = 0, P = 0, kind = 0;
  bool sparse = false, keep_y = false, sb_sparse = false;
  bool tensor = true;  // full passes over A on the tensor cores (FP64-accurate slicing)
  int* rowE = nullptr;  // biased max exponent of each row / column of A
  int* colE = nullptr;
  int *qrowE = nullptr, *qcolE = nullptr;  // ... of Q (rows: m, columns: l_max)
  int *browE = nullptr, *bcolE = nullptr;  // ... of B (rows: l_max, columns: n)
  int *xrowE = nullptr, *xcolE = nullptr;  // scratch for the operand of orth()
  OzWorkspace oz{};
  // CUDA graphs of the set-up and of each block (index j), keyed on A and lda
  struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    const double* A = nullptr;
    int64_t lda = 0;
    int dtype = LRA_F64;
    int nev0 = 0;            // first profiling event index it records
    int nev = 0;             // profiling events the graph records
    std::vector<int> phase;  // ... and their phases
    uint64_t launches = 0;   // kernel launches it holds
  };
  bool graphs = true;
  bool mixed = false;       // LRA_FLAG_MIXED: reduced digits in the sketch and power passes
  bool own_stream = false;  // st created by lra_create (the caller passed none)
  GraphSlot gpre;
  std::vector<GraphSlot> gblock;
  // the same for runs on the second host-copy buffer (lra_farpca_host_prefetch), so
  // that alternating buffers do not re-capture
  GraphSlot gpre_alt;
  std::vector<GraphSlot> gblock_alt;
  // A cut into digit images: [0] row-scaled (A X), [1] column-scaled (A^T X)
  uint8_t* ximg[2] = {nullptr, nullptr};
  bool ximg_ready = false;
  int cap = 0;  // entries per Omega column in the sparse structure
  OmegaSpec os{};
  int64_t nblk_max = 0, lmax = 0, ldq = 0, ldb = 0, lds = 0, ldf = 0, ldod = 0;

  double *Q = nullptr, *B = nullptr, *Yk = nullptr;
  double *S0 = nullptr, *Yb = nullptr, *T1 = nullptr, *Tmp = nullptr;
  double *W = nullptr, *G = nullptr, *Wt = nullptr;
  double *F = nullptr, *BOm = nullptr;
  double *z = nullptr, *zB = nullptr, *wvec = nullptr;
  double* ws = nullptr;
  int64_t ws_elems = 0;
  double* astat = nullptr;  // per-(512-row block, column) sums of squares of A
  double *gram = nullptr, *Rinv = nullptr;
  int* dead = nullptr;  // dependent columns of a power-step panel (LRA_MAX_B ints)
  // device flags: [0] the last Cholesky's Gram within 2^-40 of I (chol_inv's near);
  // [1] the last second projection taken in FP32 (project_fp32's taken)
  int* near = nullptr;
  double *colsq = nullptr, *colsum = nullptr, *scal = nullptr;
  int* flags = nullptr;
  int *om_counts = nullptr, *om_rows = nullptr;
  double *om_vals = nullptr, *om_dense = nullptr;
  // lra_sketch / lra_copy_omega scratch (grown on demand)
  int *sk_counts = nullptr, *sk_rows = nullptr;
  double* sk_vals = nullptr;
  int64_t sk_entries = 0, sk_cols = 0;
  double* A_host_copy = nullptr;  // device copy of A for lra_farpca_host
  double* A_host_copy2 = nullptr;  // ... its second buffer (prefetch of the next A)
  // the prefetch in flight or done: host source, its ld and element type, the
  // buffer (0: A_host_copy, 1: A_host_copy2) and the event its copies complete
  const void* pref_host = nullptr;
  int64_t pref_lda = 0;
  int pref_dtype = LRA_F64, pref_buf = 0;
  bool pref_valid = false;
  cudaEvent_t pref_ev = nullptr;
  // lra_farpca_host copies A in column chunks on several streams (copy engines)
  static constexpr int NCOPY = 4;
  cudaStream_t cst[NCOPY] = {};
  cudaEvent_t cev[NCOPY] = {};
  cudaEvent_t cstart = nullptr;
  Pinned* hp = nullptr;

  // phase timing (LRA_FLAG_PROFILE)
  static constexpr int NEV = 96;
  bool prof = false;
  cudaEvent_t ev0[NEV] = {}, ev1[NEV] = {};
  int ev_phase[NEV] = {};
  int nev = 0, cur_phase = 0;
  double phase_ms[LRA_NUM_PHASES] = {};
  int64_t phase_calls[LRA_NUM_PHASES] = {};

  // lra_svd: workspace for l <= svd_cap columns (grown on demand)
  struct SvdWs {
    int64_t cap = 0;
    double *Bt = nullptr, *G = nullptr, *C0 = nullptr, *C1 = nullptr, *V = nullptr;
    double *Vs = nullptr, *W = nullptr, *sigma = nullptr, *U = nullptr, *Vout = nullptr;
    double* vinv = nullptr;
    int *perm = nullptr, *info = nullptr, *btrowE = nullptr, *btcolE = nullptr, *qrowE = nullptr;
    unsigned* bar = nullptr;
  } svd;

  bool dry = false;     // lra_workspace_bytes: count allocations, make none
  bool pool = false;    // LRA_FLAG_POOL: stream-ordered allocations
  int64_t bytes = 0;    // device bytes allocated so far
  bool run_ok = false;  // the last lra_farpca_run completed (any non-negative status)
  int a_dtype = LRA_F64;  // element type of the A of the current run
  int32_t status = LRA_OK;
  int64_t rank = 0, blocks = 0;
  double E = 0.0, normA2 = 0.0;
  std::string err;
};

namespace {

lra_status fail(lra_ctx* c, lra_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CK(expr)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? LRA_ERR_OOM : LRA_ERR_CUDA,           \
                  "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define TRY(expr)                         \
  do {                                    \
    lra_status s_ = (expr);               \
    if (s_ < 0) return s_;                \
  } while (0)

// Device memory of a context: cudaMalloc, or with LRA_FLAG_POOL the device's
// stream-ordered pool on the context's stream (freeing it then synchronises
// nothing but that stream).  A dry context (lra_workspace_bytes) only counts.
template <class T>
cudaError_t dalloc(lra_ctx* ctx, T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) return cudaSuccess;
  const size_t bytes = (size_t)count * sizeof(T);
  ctx->bytes += (int64_t)bytes;
  if (ctx->dry) return cudaSuccess;
  if (ctx->pool) return cudaMallocAsync((void**)p, bytes, ctx->st);
  return cudaMalloc((void**)p, bytes);
}

void dfree(lra_ctx* ctx, void* p) {
  if (!p) return;
  if (ctx->pool)
    cudaFreeAsync(p, ctx->st);
  else
    cudaFree(p);
}

double default_p(int kind, int64_t n, int zeta) {
  if (kind == LRA_OMEGA_SPARSE_GAUSSIAN && zeta > 0) return (double)zeta / (double)n;
  if (kind == LRA_OMEGA_STD_BERNOULLI) return std::max(1e-3, log((double)n) / (double)n);
  return std::max(1e-3, 10.0 / (double)n);
}

lra_status check_params(lra_ctx* ctx, int64_t m, int64_t n, const lra_params* p) {
  if (m < 1 || n < 1 || m > INT32_MAX || n > INT32_MAX)
    return fail(ctx, LRA_ERR_INVALID_ARG, "m and n must lie in [1, 2^31)");
  const int64_t mn = std::min(m, n);
  if (p->b < 1 || p->b > LRA_MAX_B || p->b > mn)
    return fail(ctx, LRA_ERR_INVALID_ARG, "b must lie in [1, min(m, n, %d)]", LRA_MAX_B);
  if (p->P < 0 || p->P > LRA_MAX_P)
    return fail(ctx, LRA_ERR_INVALID_ARG, "P must lie in [0, %d]", LRA_MAX_P);
  if (p->kind < 0 || p->kind > LRA_OMEGA_BERNOULLI)
    return fail(ctx, LRA_ERR_INVALID_ARG, "unknown Omega kind %d", p->kind);
  if (p->k < 0 || p->k > mn) return fail(ctx, LRA_ERR_INVALID_ARG, "k must lie in [0, min(m, n)]");
  if (p->k == 0 && !(p->eps > 0.0 && isfinite(p->eps)))
    return fail(ctx, LRA_ERR_INVALID_ARG, "eps must be finite and > 0 when k == 0");
  if (p->k > 0 && (p->k + p->b - 1) / p->b * p->b > mn)
    return fail(ctx, LRA_ERR_INVALID_ARG, "ceil(k/b) b exceeds min(m, n)");
  if (p->kind == LRA_OMEGA_SPARSE_SIGN && (p->zeta < 1 || p->zeta > n || p->zeta > LRA_MAX_ZETA))
    return fail(ctx, LRA_ERR_INVALID_ARG, "zeta must lie in [1, min(n, %d)]", LRA_MAX_ZETA);
  if (p->kind != LRA_OMEGA_SPARSE_SIGN && p->zeta < 0)
    return fail(ctx, LRA_ERR_INVALID_ARG, "zeta must be >= 0");
  if (!(p->p >= 0.0 && p->p < 1.0)) return fail(ctx, LRA_ERR_INVALID_ARG, "p must lie in [0, 1)");
  if (p->max_blocks < 0) return fail(ctx, LRA_ERR_INVALID_ARG, "max_blocks must be >= 0");
  if ((int64_t)p->max_blocks * p->b > mn)
    return fail(ctx, LRA_ERR_INVALID_ARG, "max_blocks * b exceeds min(m, n)");
  if (p->flags & ~(LRA_FLAG_KEEP_Y | LRA_FLAG_PROFILE | LRA_FLAG_FP64_SIMT | LRA_FLAG_NO_A_DIGITS |
                   LRA_FLAG_NO_GRAPHS | LRA_FLAG_MIXED | LRA_FLAG_POOL))
    return fail(ctx, LRA_ERR_INVALID_ARG, "unknown flags");
  return LRA_OK;
}

lra_status check_matrix(lra_ctx* ctx, const lra_matrix* A, bool allow_f32 = false) {
  if (!A || !A->data) return fail(ctx, LRA_ERR_INVALID_ARG, "A is NULL");
  if (A->m != ctx->m || A->n != ctx->n)
    return fail(ctx, LRA_ERR_INVALID_ARG, "A is %lld x %lld, context expects %lld x %lld",
                (long long)A->m, (long long)A->n, (long long)ctx->m, (long long)ctx->n);
  if (A->lda < A->m) return fail(ctx, LRA_ERR_INVALID_ARG, "lda < m");
  if (A->dtype == LRA_F32 && !allow_f32)
    return fail(ctx, LRA_ERR_UNSUPPORTED, "this entry point takes LRA_F64 matrices only");
  if (A->dtype != LRA_F64 && A->dtype != LRA_F32)
    return fail(ctx, LRA_ERR_INVALID_ARG, "unknown dtype %d", (int)A->dtype);
  return LRA_OK;
}

// ---- device steps ---------------------------------------------------------

lra_status gemm(lra_ctx* ctx, bool trans, int64_t P, int64_t N, int64_t K, double alpha,
                const double* X, int64_t ldx, const double* Y, int64_t ldy, double beta, double* C,
                int64_t csp, int64_t csc) {
  CK(dgemm(trans, P, N, K, alpha, X, ldx, Y, ldy, beta, GemmOut{C, csp, csc}, ctx->ws,
           ctx->ws_elems, ctx->st));
  return LRA_OK;
}

// A full pass over A: C = alpha op(A) Y + beta C (op(A) = A^T when trans).  Inside
// lra_farpca_run the digit images of A, once cut, replace A itself.
// power: a sketch or power-step pass, which the mixed precision form runs reduced.
// ydig1: Y holds 0 and +-2^k per column only (the +-1/2 and 0/1 test matrices), so
// the image-fed pass multiplies its first digit plane alone (the same result).
lra_status dense(lra_ctx* ctx, bool trans, int64_t N, double alpha, const double* A, int64_t lda,
                 const double* Y, int64_t ldy, double beta, double* C, int64_t csp, int64_t csc,
                 bool power = false, bool ydig1 = false) {
  const int64_t P = trans ? ctx->n : ctx->m, K = trans ? ctx->m : ctx->n;
  if (!ctx->tensor || K > oz_max_k())
    return gemm(ctx, trans, P, N, K, alpha, A, lda, Y, ldy, beta, C, csp, csc);
  if (ctx->ximg_ready) {
    CK(ozgemm_img(P, N, K, alpha, ctx->ximg[trans ? 1 : 0], trans ? ctx->colE : ctx->rowE, Y, ldy,
                  beta, GemmOut{C, csp, csc}, ctx->oz, ctx->flags, ctx->st, power && ctx->mixed,
                  ydig1));
    return LRA_OK;
  }
  CK(ozgemm(trans, P, N, K, alpha, A, lda, trans ? ctx->colE : ctx->rowE, Y, ldy, beta,
            GemmOut{C, csp, csc}, ctx->oz, ctx->flags, ctx->st));
  return LRA_OK;
}

lra_status a_exponents(lra_ctx* ctx, const double* A, int64_t lda) {
  if (ctx->tensor)
    CK(oz_rowcol_exponents(A, lda, ctx->m, ctx->n, ctx->rowE, ctx->colE, ctx->st));
  return LRA_OK;
}

// C = alpha op(X) Y + beta C with the context's engine.  xE: biased max exponent
// of each row of op(X); the tensor engine needs it (NULL selects the FP64 cores).
lra_status mm(lra_ctx* ctx, bool trans, int64_t P, int64_t N, int64_t K, double alpha,
              const double* X, int64_t ldx, const int* xE, const double* Y, int64_t ldy,
              double beta, double* C, int64_t csp, int64_t csc, const int* yE_known = nullptr) {
  if (!ctx->tensor || !xE || K > oz_max_k())
    return gemm(ctx, trans, P, N, K, alpha, X, ldx, Y, ldy, beta, C, csp, csc);
  if (P <= 0 || N <= 0) return LRA_OK;
  if (K <= 0) return LRA_OK;
  CK(ozgemm(trans, P, N, K, alpha, X, ldx, xE, Y, ldy, beta, GemmOut{C, csp, csc}, ctx->oz,
            ctx->flags, ctx->st, yE_known));
  return LRA_OK;
}

// S = X^T X (b x b) and Tmp-style right multiplication X R^{-1}, both on the
// context's engine; exponents of X computed on the fly.
lra_status gram(lra_ctx* ctx, const double* X, int64_t ldx, int64_t rows) {
  const int b = ctx->b;
  const int* xE = nullptr;
  if (ctx->tensor) {
    CK(oz_rowcol_exponents(X, ldx, rows, b, nullptr, ctx->xcolE, ctx->st));
    xE = ctx->xcolE;
  }
  // X^T X: the right operand's column exponents are the left operand's row exponents
  return mm(ctx, true, b, b, rows, 1.0, X, ldx, xE, X, ldx, 0.0, ctx->gram, 1, b, xE);
}

// The Gram S = X^T X and its Cholesky factor R^{-1} (into ctx->Rinv): on the tensor
// engine in one launch after the product (the fused fixup + Cholesky); dead as
// for chol_inv; near: ctx->near[0] records whether S is within 2^-40 of I.
lra_status gram_chol(lra_ctx* ctx, const double* X, int64_t ldx, int64_t rows, int* dead,
                     bool near = false) {
  const int b = ctx->b;
  int* nr = near ? ctx->near : nullptr;
  if (!ctx->tensor || rows > oz_max_k()) {
    TRY(gram(ctx, X, ldx, rows));
    CK(chol_inv(ctx->gram, b, PIVOT_TAU, ctx->Rinv, ctx->flags, ctx->st, dead, nr));
    return LRA_OK;
  }
  CK(oz_rowcol_exponents(X, ldx, rows, b, nullptr, ctx->xcolE, ctx->st));
  const CholJob job{ctx->Rinv, dead, ctx->oz.count, PIVOT_TAU, nr};
  // X^T X: the right operand's column exponents are the left operand's row exponents
  CK(ozgemm(true, b, b, rows, 1.0, X, ldx, ctx->xcolE, X, ldx, 0.0, GemmOut{ctx->gram, 1, b}, ctx->oz,
            ctx->flags, ctx->st, ctx->xcolE, &job));
  return LRA_OK;
}

lra_status right_apply_rinv(lra_ctx* ctx, const double* X, int64_t ldx, int64_t rows, double* out,
                            int64_t ldo) {
  const int b = ctx->b;
  const int* xE = nullptr;
  if (ctx->tensor) {
    CK(oz_rowcol_exponents(X, ldx, rows, b, ctx->xrowE, nullptr, ctx->st));
    xE = ctx->xrowE;
  }
  return mm(ctx, false, rows, b, b, 1.0, X, ldx, xE, ctx->Rinv, b, 0.0, out, 1, ldo);
}

// The second pass of CholQR2: the Gram of X = Tmp (the first pass's Q factor) and
// out = X R^{-1}.  The Gram is normally within the first pass's loss of
// orthogonality of I; when every entry of S - I is within 2^-40 the product is
// X + X (R^{-1} - I) with the small correction in FP32 (rinv_near_identity),
// otherwise the FP64-accurate product.  The choice is made on the device (the
// Cholesky's flag): both are issued, and the one not chosen does nothing.
lra_status second_pass(lra_ctx* ctx, const double* X, int64_t ldx, int64_t rows, double* out,
                       int64_t ldo) {
  const int b = ctx->b;
  if (!ctx->tensor || rows > oz_max_k()) {
    TRY(gram_chol(ctx, X, ldx, rows, nullptr));
    return right_apply_rinv(ctx, X, ldx, rows, out, ldo);
  }
  TRY(gram_chol(ctx, X, ldx, rows, nullptr, true));
  CK(rinv_near_identity(X, ldx, rows, b, ctx->Rinv, ctx->near, out, ldo, ctx->st));
  CK(oz_rowcol_exponents(X, ldx, rows, b, ctx->xrowE, nullptr, ctx->st, false, ctx->near));
  CK(ozgemm(false, rows, b, b, 1.0, X, ldx, ctx->xrowE, ctx->Rinv, b, 0.0, GemmOut{out, 1, ldo},
            ctx->oz, ctx->flags, ctx->st, nullptr, nullptr, ctx->near));
  return LRA_OK;
}

// out (rows x b, ld ldo) = Q factor of X (rows x b, ld ldx), CholQR2.
lra_status orth(lra_ctx* ctx, const double* X, int64_t ldx, int64_t rows, double* out,
                int64_t ldo) {
  TRY(gram_chol(ctx, X, ldx, rows, nullptr));
  TRY(right_apply_rinv(ctx, X, ldx, rows, ctx->Tmp, ctx->lds));
  return second_pass(ctx, ctx->Tmp, ctx->lds, rows, out, ldo);
}

// The basis G of the power-step panel W of block j, power step s (the eigSVD step
// of Alg. 1).  A numerically dependent column of W does not end the run: the first
// CholQR pass skips its pivot, the column of W R^{-1} is replaced by a fixed
// random direction (+-1/sqrt(rows), TAG_FILL stream), and the second pass
// orthonormalises the completed panel.  Without a dependent column this is orth().
lra_status orth_panel(lra_ctx* ctx, const double* X, int64_t ldx, int64_t rows, double* out,
                      int64_t ldo, int64_t j, int s) {
  const int b = ctx->b;
  TRY(gram_chol(ctx, X, ldx, rows, ctx->dead));
  TRY(right_apply_rinv(ctx, X, ldx, rows, ctx->Tmp, ctx->lds));
  CK(fill_dead(ctx->Tmp, ctx->lds, rows, b, ctx->dead, ctx->os.k0, ctx->os.k1, j, s, ctx->st));
  return second_pass(ctx, ctx->Tmp, ctx->lds, rows, out, ldo);
}

lra_status make_omega(lra_ctx* ctx, int64_t j) {
  if (ctx->sparse)
    CK(omega_sparse(ctx->os, j, 1, ctx->cap, ctx->om_counts, ctx->om_rows, ctx->om_vals, ctx->flags,
                    ctx->st));
  else
    CK(omega_dense(ctx->os, j, 1, ctx->om_dense, ctx->ldod, ctx->st));
  return LRA_OK;
}

// out (rows_x x b) = X Omega_j (minus the standardized-Bernoulli shift when sparse);
// X is A (x_is_A) or the rows of B.
lra_status apply_omega(lra_ctx* ctx, const double* X, int64_t ldx, int64_t rows_x, double* out,
                       int64_t ldo, const double* shift, bool x_is_A) {
  if (ctx->sparse) {
    CK(gather_sketch(X, x_is_A ? ctx->a_dtype : LRA_F64, ldx, rows_x, ctx->om_counts, ctx->om_rows,
                     ctx->om_vals, ctx->cap, ctx->b, out, ldo, shift, ctx->flags, ctx->st));
    return LRA_OK;
  }
  if (x_is_A) {
    // the standardized Bernoulli matrix at p = 1/2 (entries B - p = +-1/2) and the
    // Bernoulli matrix (0 / 1) are one digit each
    const bool one_digit = (ctx->kind == LRA_OMEGA_STD_BERNOULLI && ctx->os.p == 0.5) ||
                           ctx->kind == LRA_OMEGA_BERNOULLI;
    return dense(ctx, false, ctx->b, 1.0, X, ldx, ctx->om_dense, ctx->ldod, 0.0, out, 1, ldo, true,
                 one_digit);
  }
  return mm(ctx, false, rows_x, ctx->b, ctx->n, 1.0, X, ldx, ctx->browE, ctx->om_dense, ctx->ldod, 0.0,
            out, 1, ldo);
}

lra_status compute_z(lra_ctx* ctx, const double* A, int64_t lda) {
  // z = A w, w = p 1 (Alg. 2 step 2)
  CK(fill(ctx->wvec, ctx->n, ctx->n, 1, ctx->os.p, ctx->st));
  return dense(ctx, false, 1, 1.0, A, lda, ctx->wvec, ctx->n, 0.0, ctx->z, 1, ctx->m);
}

// Phase timing: events recorded on the context's stream around each phase,
// read back at the per-block synchronisation point.
lra_status prof_flush(lra_ctx* ctx) {
  if (!ctx->prof || ctx->nev == 0) return LRA_OK;
  CK(cudaStreamSynchronize(ctx->st));
  for (int i = 0; i < ctx->nev; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0[i], ctx->ev1[i]));
    ctx->phase_ms[ctx->ev_phase[i]] += ms;
    ctx->phase_calls[ctx->ev_phase[i]] += 1;
  }
  ctx->nev = 0;
  return LRA_OK;
}

// Records ev on the context's stream.  Inside a graph capture the record must be
// external, so that the graph records the event at every replay (a plain record
// would only order the capture); outside a capture the flag is not accepted.
cudaError_t record(lra_ctx* ctx, cudaEvent_t ev) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(ctx->st, &cs);
  if (e != cudaSuccess) return e;
  if (cs == cudaStreamCaptureStatusActive)
    return cudaEventRecordWithFlags(ev, ctx->st, cudaEventRecordExternal);
  return cudaEventRecord(ev, ctx->st);
}

lra_status prof_begin(lra_ctx* ctx, int phase) {
  if (!ctx->prof) return LRA_OK;
  if (ctx->nev == lra_ctx::NEV) TRY(prof_flush(ctx));
  CK(record(ctx, ctx->ev0[ctx->nev]));
  ctx->cur_phase = phase;
  return LRA_OK;
}

lra_status prof_end(lra_ctx* ctx) {
  if (!ctx->prof) return LRA_OK;
  CK(record(ctx, ctx->ev1[ctx->nev]));
  ctx->ev_phase[ctx->nev] = ctx->cur_phase;
  ctx->nev += 1;
  return LRA_OK;
}

#define PHASE(ph, body)            \
  do {                             \
    TRY(prof_begin(ctx, (ph)));    \
    body;                          \
    TRY(prof_end(ctx));            \
  } while (0)

lra_status read_record(lra_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->hp->v, ctx->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(&ctx->hp->flags, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return prof_flush(ctx);
}

// Runs body on the context's stream as a CUDA graph: captured on first use (and
// again when A or lda change), replayed afterwards.  The host-side counters that
// body advances while it issues work (profiling events, kernel launches) advance
// by the graph's amounts at every replay.  A capture always ends, also on error,
// so the stream stays usable.
template <typename F>
lra_status captured(lra_ctx* ctx, lra_ctx::GraphSlot& gs, const double* A, int64_t lda, F&& body) {
  if (!gs.exec || gs.A != A || gs.lda != lda || gs.dtype != ctx->a_dtype || gs.nev0 != ctx->nev) {
    if (gs.exec) {
      cudaGraphExecDestroy(gs.exec);
      gs.exec = nullptr;
    }
    const int nev0 = ctx->nev;
    const uint64_t l0 = g_launches.load();
    CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
    const lra_status s = body();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->st, &g);
    const uint64_t launches = g_launches.load() - l0;
    g_launches.fetch_sub(launches);
    const int nev = ctx->nev - nev0;
    ctx->nev = nev0;
    if (s != LRA_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      if (s != LRA_OK) return s;
      return fail(ctx, LRA_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    const cudaError_t ei = cudaGraphInstantiate(&gs.exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      gs.exec = nullptr;
      return fail(ctx, LRA_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ei));
    }
    gs.A = A;
    gs.lda = lda;
    gs.dtype = ctx->a_dtype;
    gs.nev0 = nev0;
    gs.nev = nev;
    gs.phase.assign(ctx->ev_phase + nev0, ctx->ev_phase + nev0 + nev);
    gs.launches = launches;
  }
  CK(cudaGraphLaunch(gs.exec, ctx->st));
  // the graph records events nev .. nev + gs.nev - 1 (the indices of its capture)
  for (int i = 0; i < gs.nev; ++i) ctx->ev_phase[ctx->nev + i] = gs.phase[i];
  ctx->nev += gs.nev;
  g_launches.fetch_add(gs.launches);
  return LRA_OK;
}

template <typename F>
lra_status issue(lra_ctx* ctx, lra_ctx::GraphSlot& gs, const double* A, int64_t lda, F&& body) {
  if (ctx->graphs) return captured(ctx, gs, A, lda, body);
  return body();
}

// A: column-major m x n of element type dtype.  FP32 entries are converted
// exactly to FP64 where they are read (the statistics pass, the digit cut and
// the sparse gather); nothing else reads A, so a run on FP32 data computes the
// same bits as a run on its FP64 conversion.
lra_status run(lra_ctx* ctx, const void* Av, int64_t lda, int dtype) {
  if (dtype == LRA_F32 && !(ctx->tensor && ctx->ximg[0] && ctx->ximg[1]))
    return fail(ctx, LRA_ERR_UNSUPPORTED,
                "LRA_F32 input needs the tensor engine with digit images (no LRA_FLAG_FP64_SIMT, "
                "no LRA_FLAG_NO_A_DIGITS, and room for the images)");
  ctx->a_dtype = dtype;
  const double* A = (const double*)Av;  // dereferenced as double only when dtype is LRA_F64
  // the digit images describe this run's A only: invalid on every way out
  struct ImageScope {
    lra_ctx* c;
    ~ImageScope() { c->ximg_ready = false; }
  } image_scope{ctx};
  const int64_t m = ctx->m, n = ctx->n, lds = ctx->lds, ldq = ctx->ldq, ldb = ctx->ldb,
                ldf = ctx->ldf;
  const int b = ctx->b, P = ctx->P;
  ctx->status = LRA_OK;
  ctx->run_ok = false;
  ctx->rank = ctx->blocks = 0;
  ctx->E = ctx->normA2 = 0.0;
  CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int), ctx->st));
  // ||A||_F^2 (Alg. 1 step 1); the tensor engine takes the exponents of A's rows
  // and columns in the same pass.  With digit images, the row-scaled cut reads
  // every entry of A anyway and sums the squares there (its FP64 pipe is idle),
  // so this pass takes the exponents alone and ||A||_F^2 is read after the cut.
  const bool images = ctx->tensor && ctx->ximg[0] && ctx->ximg[1];
  PHASE(LRA_PHASE_INDICATOR, {
    if (ctx->tensor)
      CK(a_stats(Av, dtype, lda, m, n, images ? nullptr : ctx->astat, ctx->colsq, ctx->colE,
                 ctx->rowE, ctx->st));
    else
      CK(col_sums(A, lda, m, n, ctx->colsq, nullptr, ctx->st));
    if (!images) CK(total(ctx->colsq, n, ctx->scal, ctx->st));
  });
  double normA2 = 0.0;
  // 1: ||A||_F^2 read and usable; 0: the run is over (A = 0, or an error)
  auto take_norm = [&](lra_status& r) -> int {
    r = read_record(ctx);
    if (r != LRA_OK) return 0;
    normA2 = ctx->hp->v[0];
    if (!isfinite(normA2)) {
      r = fail(ctx, LRA_ERR_INVALID_ARG, "A has non-finite entries");
      return 0;
    }
    ctx->normA2 = ctx->E = normA2;
    if (normA2 == 0.0) {
      ctx->E = 0.0;
      ctx->run_ok = true;
      r = LRA_OK;
      return 0;
    }
    return 1;
  };
  lra_status norm_status = LRA_OK;
  if (!images && !take_norm(norm_status)) return norm_status;
  // set-up: exponents of A, its digit images, z = A (p 1) for the shifted sketch
  ctx->ximg_ready = images;  // stream order puts the cut before every pass that reads it
  // runs on the prefetch buffer keep their own graphs
  const bool alt = ctx->A_host_copy2 && (const void*)A == (const void*)ctx->A_host_copy2;
  lra_ctx::GraphSlot& gpre = alt ? ctx->gpre_alt : ctx->gpre;
  std::vector<lra_ctx::GraphSlot>& gblock = alt ? ctx->gblock_alt : ctx->gblock;
  TRY(issue(ctx, gpre, A, lda, [&]() -> lra_status {
    if (images) {
      PHASE(LRA_PHASE_CUT, {
        CK(oz_cut_x(false, m, n, Av, dtype, lda, ctx->rowE, ctx->ximg[0], ctx->oz.ctas, ctx->st,
                    ctx->astat));
        CK(oz_cut_x(true, n, m, Av, dtype, lda, ctx->colE, ctx->ximg[1], ctx->oz.ctas, ctx->st));
      });
      PHASE(LRA_PHASE_INDICATOR,
            CK(total(ctx->astat, oz_cut_ctas(m, n, ctx->oz.ctas), ctx->scal, ctx->st)));
    }
    if (ctx->tensor) {
      CK(cudaMemsetAsync(ctx->qrowE, 0, m * sizeof(int), ctx->st));
      CK(cudaMemsetAsync(ctx->bcolE, 0, n * sizeof(int), ctx->st));
    }
    if (ctx->sb_sparse) PHASE(LRA_PHASE_SKETCH, TRY(compute_z(ctx, A, lda)));
    return LRA_OK;
  }));
  if (images && !take_norm(norm_status)) return norm_status;
  const double thr = ctx->prm.eps * ctx->prm.eps * normA2;
  const bool fixed_rank = ctx->prm.k > 0;
  double E = normA2;
  int32_t status = fixed_rank ? LRA_OK : LRA_NOT_CONVERGED;
  for (int64_t j = 0; j < ctx->nblk_max; ++j) {
    if ((int64_t)gblock.size() <= j) gblock.resize(j + 1);
    TRY(issue(ctx, gblock[j], A, lda, [&]() -> lra_status {
      const int64_t l = j * b;
      PHASE(LRA_PHASE_OMEGA, TRY(make_omega(ctx, j)));
      PHASE(LRA_PHASE_SKETCH,
            TRY(apply_omega(ctx, A, lda, m, ctx->S0, lds, ctx->sb_sparse ? ctx->z : nullptr, true)));
      double* Y = ctx->S0;
      if (P >= 1) {
        PHASE(LRA_PHASE_DENSE,
            TRY(dense(ctx, true, b, 1.0, A, lda, ctx->S0, lds, 0.0, ctx->W, 1, lds, true)));
        if (l > 0) {
          PHASE(LRA_PHASE_DEFLATE, {
            TRY(apply_omega(ctx, ctx->B, ldb, l, ctx->BOm, ldf, ctx->sb_sparse ? ctx->zB : nullptr,
                            false));
            TRY(mm(ctx, true, n, b, l, -1.0, ctx->B, ldb, ctx->bcolE, ctx->BOm, ldf, 1.0, ctx->W, 1,
                   lds));
          });
        }
        PHASE(LRA_PHASE_ORTH, TRY(orth_panel(ctx, ctx->W, lds, n, ctx->G, lds, j, 0)));
        for (int s = 1; s < P; ++s) {
          PHASE(LRA_PHASE_DENSE,
                TRY(dense(ctx, false, b, 1.0, A, lda, ctx->G, lds, 0.0, ctx->T1, 1, lds, true)));
          PHASE(LRA_PHASE_DENSE,
                TRY(dense(ctx, true, b, 1.0, A, lda, ctx->T1, lds, 0.0, ctx->W, 1, lds, true)));
          if (l > 0) {
            PHASE(LRA_PHASE_DEFLATE, {
              TRY(mm(ctx, false, l, b, n, 1.0, ctx->B, ldb, ctx->browE, ctx->G, lds, 0.0, ctx->BOm, 1,
                     ldf));
              TRY(mm(ctx, true, n, b, l, -1.0, ctx->B, ldb, ctx->bcolE, ctx->BOm, ldf, 1.0, ctx->W, 1,
                     lds));
            });
          }
          PHASE(LRA_PHASE_ORTH, TRY(orth_panel(ctx, ctx->W, lds, n, ctx->G, lds, j, s)));
        }
        PHASE(LRA_PHASE_DENSE,
              TRY(dense(ctx, false, b, 1.0, A, lda, ctx->G, lds, 0.0, ctx->Yb, 1, lds, true)));
        Y = ctx->Yb;
      }
      if (ctx->keep_y)
        CK(cudaMemcpy2DAsync(ctx->Yk + l * ldq, ldq * sizeof(double), Y, lds * sizeof(double),
                             m * sizeof(double), b, cudaMemcpyDeviceToDevice, ctx->st));
      if (l > 0) {
        PHASE(LRA_PHASE_PROJECT, {
          for (int pass = 0; pass < 2; ++pass) {
            TRY(mm(ctx, true, l, b, m, 1.0, ctx->Q, ldq, ctx->qcolE, Y, lds, 0.0, ctx->F, 1, ldf));
            if (pass == 1 && ctx->tensor && m <= oz_max_k() && l <= 4096) {
              // F = Q^T Y is now of the order of Y's rounding: the update in FP32 when
              // small enough (decided on the device), else the FP64-accurate product
              // (whose scan of F's exponents may skip for l <= 4096); the product just
              // made left Y's column exponents in oz.yE
              CK(project_fp32(ctx->Q, ldq, m, l, ctx->F, ldf, b, ctx->oz.yE, Y, lds, ctx->near + 1,
                              ctx->st));
              CK(ozgemm(false, m, b, l, -1.0, ctx->Q, ldq, ctx->qrowE, ctx->F, ldf, 1.0,
                        GemmOut{Y, 1, lds}, ctx->oz, ctx->flags, ctx->st, nullptr, nullptr,
                        ctx->near + 1));
            } else {
              TRY(mm(ctx, false, m, b, l, -1.0, ctx->Q, ldq, ctx->qrowE, ctx->F, ldf, 1.0, Y, 1,
                     lds));
            }
          }
        });
      }
      double* Qj = ctx->Q + l * ldq;
      PHASE(LRA_PHASE_ORTH, TRY(orth(ctx, Y, lds, m, Qj, ldq)));
      PHASE(LRA_PHASE_DENSE, TRY(dense(ctx, true, b, 1.0, A, lda, Qj, ldq, 0.0, ctx->Wt, 1, lds)));
      PHASE(LRA_PHASE_INDICATOR, {
        CK(col_sums(ctx->Wt, lds, n, b, ctx->colsq, ctx->sb_sparse ? ctx->colsum : nullptr, ctx->st));
        CK(total(ctx->colsq, b, ctx->scal + 1, ctx->st));
        CK(append_rows(ctx->Wt, lds, n, b, ctx->B, ldb, l, ctx->colsum, ctx->os.p,
                       ctx->sb_sparse ? ctx->zB : nullptr, ctx->st));
        if (ctx->tensor) {
          // Q_j: its column maxima, and the running row maxima of Q
          CK(oz_rowcol_exponents(Qj, ldq, m, b, ctx->qrowE, ctx->qcolE + l, ctx->st, true));
          // B_j = Wt^T: row maxima of B_j are Wt's column maxima; B's column maxima grow
          CK(oz_rowcol_exponents(ctx->Wt, lds, n, b, ctx->bcolE, ctx->browE + l, ctx->st, true));
        }
      });
      return LRA_OK;
    }));
    TRY(read_record(ctx));
    const int fl = ctx->hp->flags;
    if (fl & FLAG_TIMEOUT) return fail(ctx, LRA_ERR_TIMEOUT, "a device wait timed out");
    if (fl & FLAG_OMEGA_CAP)
      return fail(ctx, LRA_ERR_INVALID_ARG, "fixed-zeta draws exhausted (zeta too close to n)");
    if (fl & FLAG_BREAKDOWN) {
      status = LRA_BREAKDOWN;
      break;
    }
    E -= ctx->hp->v[1];
    ctx->blocks = j + 1;
    ctx->rank = (j + 1) * b;
    ctx->E = E;
    if (!fixed_rank && E < thr) {
      status = LRA_OK;
      break;
    }
  }
  ctx->status = status;
  ctx->run_ok = true;
  return (lra_status)status;
}

lra_status ensure_sketch_scratch(lra_ctx* ctx, int64_t cols, int cap) {
  const int64_t entries = cols * cap;
  if (cols <= ctx->sk_cols && entries <= ctx->sk_entries) return LRA_OK;
  dfree(ctx, ctx->sk_counts);
  dfree(ctx, ctx->sk_rows);
  dfree(ctx, ctx->sk_vals);
  ctx->sk_counts = nullptr;
  ctx->sk_rows = nullptr;
  ctx->sk_vals = nullptr;
  ctx->sk_cols = ctx->sk_entries = 0;
  CK(dalloc(ctx, &ctx->sk_counts, cols));
  CK(dalloc(ctx, &ctx->sk_rows, entries));
  CK(dalloc(ctx, &ctx->sk_vals, entries));
  ctx->sk_cols = cols;
  ctx->sk_entries = entries;
  return LRA_OK;
}

void svd_free(lra_ctx* ctx) {
  auto& w = ctx->svd;
  void* ptrs[] = {w.Bt, w.G,    w.C0,   w.C1,     w.V,      w.Vs,     w.W,    w.sigma,
                  w.U,  w.Vout, w.perm, w.info,   w.btrowE, w.btcolE, w.qrowE, w.bar, w.vinv};
  for (void* p : ptrs) dfree(ctx, p);
  w = lra_ctx::SvdWs{};
}

// Workspace of lra_svd for l columns (kept, and grown, across calls).
lra_status svd_alloc(lra_ctx* ctx, int64_t l) {
  auto& w = ctx->svd;
  if (w.cap >= l) return LRA_OK;
  svd_free(ctx);
  const int64_t lp = eig_padded(l), m = ctx->m, n = ctx->n;
  CK(dalloc(ctx, &w.Bt, n * l));
  CK(dalloc(ctx, &w.G, l * l));
  CK(dalloc(ctx, &w.C0, lp * lp));
  CK(dalloc(ctx, &w.C1, std::max<int64_t>(lp * lp, 3 * lp)));  // the Jacobi snapshot
  CK(dalloc(ctx, &w.V, lp * lp));
  CK(dalloc(ctx, &w.Vs, l * l));
  CK(dalloc(ctx, &w.W, l * l));
  CK(dalloc(ctx, &w.sigma, l));
  CK(dalloc(ctx, &w.U, m * l));
  CK(dalloc(ctx, &w.Vout, n * l));
  CK(dalloc(ctx, &w.perm, l));
  CK(dalloc(ctx, &w.vinv, l));
  CK(dalloc(ctx, &w.info, 4));
  CK(dalloc(ctx, &w.btrowE, n));
  CK(dalloc(ctx, &w.btcolE, l));
  CK(dalloc(ctx, &w.qrowE, m));
  CK(dalloc(ctx, &w.bar, 5));
  w.cap = l;
  return LRA_OK;
}

void free_all(lra_ctx* c) {
  // a prefetch may still be copying into a buffer freed below
  for (int i = 0; i < lra_ctx::NCOPY; ++i)
    if (c->cst[i]) cudaStreamSynchronize(c->cst[i]);
  void* ptrs[] = {c->Q,      c->B,        c->Yk,     c->S0,       c->Yb,        c->T1,
                  c->Tmp,    c->W,        c->G,      c->Wt,       c->F,         c->BOm,
                  c->z,      c->zB,       c->wvec,   c->ws,       c->gram,      c->Rinv,   c->dead,   c->near,
                  c->colsq,  c->colsum,   c->scal,   c->flags,    c->om_counts, c->om_rows,
                  c->om_vals, c->om_dense, c->sk_counts, c->sk_rows, c->sk_vals, c->A_host_copy,
                  c->A_host_copy2,
                  c->rowE,   c->colE,     c->oz.yE,  c->oz.img,   c->oz.part,  c->oz.count,
                  c->qrowE,  c->qcolE,    c->browE,  c->bcolE,    c->xrowE,     c->xcolE,
                  c->ximg[0], c->ximg[1], c->astat};
  for (void* p : ptrs) dfree(c, p);
  svd_free(c);
  if (c->hp) {
    if (c->st) cudaStreamSynchronize(c->st);  // no copy into the slot may be pending
    pinned_arena().put(c->hp);
    c->hp = nullptr;
  }
  if (c->gpre.exec) cudaGraphExecDestroy(c->gpre.exec);
  if (c->gpre_alt.exec) cudaGraphExecDestroy(c->gpre_alt.exec);
  for (auto& g : c->gblock_alt)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (c->pref_ev) cudaEventDestroy(c->pref_ev);
  for (int i = 0; i < lra_ctx::NCOPY; ++i) {
    if (c->cst[i]) cudaStreamDestroy(c->cst[i]);
    if (c->cev[i]) cudaEventDestroy(c->cev[i]);
  }
  if (c->cstart) cudaEventDestroy(c->cstart);
  if (c->own_stream && c->st) {
    cudaStreamDestroy(c->st);
    c->st = nullptr;
  }
  for (auto& g : c->gblock)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (int i = 0; i < lra_ctx::NEV; ++i) {
    if (c->ev0[i]) cudaEventDestroy(c->ev0[i]);
    if (c->ev1[i]) cudaEventDestroy(c->ev1[i]);
  }
}

}  // namespace

extern "C" {

int32_t lra_version(void) { return LRA_VERSION; }

uint64_t lra_kernel_launches(void) { return g_launches.load(); }

const char* lra_status_string(int32_t s) {
  switch (s) {
    case LRA_OK: return "LRA_OK";
    case LRA_NOT_CONVERGED: return "LRA_NOT_CONVERGED";
    case LRA_BREAKDOWN: return "LRA_BREAKDOWN";
    case LRA_ERR_INVALID_ARG: return "LRA_ERR_INVALID_ARG";
    case LRA_ERR_OOM: return "LRA_ERR_OOM";
    case LRA_ERR_CUDA: return "LRA_ERR_CUDA";
    case LRA_ERR_TIMEOUT: return "LRA_ERR_TIMEOUT";
    case LRA_ERR_UNSUPPORTED: return "LRA_ERR_UNSUPPORTED";
    default: return "unknown status";
  }
}

const char* lra_last_error(const lra_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

int64_t lra_capacity(const lra_ctx* ctx) { return ctx ? ctx->lmax : -1; }

namespace {

// lra_create, or with dry = true the same sizing with every allocation only
// counted (ctx->bytes) and no CUDA object made.
lra_status create_ctx(lra_ctx** out, int64_t m, int64_t n, const lra_params* params,
                      void* cuda_stream, bool dry) {
  if (!out || !params) return LRA_ERR_INVALID_ARG;
  *out = nullptr;
  lra_ctx* ctx = new lra_ctx();
  ctx->dry = dry;
  ctx->pool = (params->flags & LRA_FLAG_POOL) != 0;
  lra_status s = check_params(ctx, m, n, params);
  if (s != LRA_OK) {
    delete ctx;
    return s;
  }
  ctx->m = m;
  ctx->n = n;
  ctx->prm = *params;
  ctx->st = (cudaStream_t)cuda_stream;
  if (!ctx->st && !dry) {
    // a blocking stream of our own: ordered with the legacy default stream like
    // NULL, but capturable into graphs
    if (cudaStreamCreate(&ctx->st) != cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return LRA_ERR_CUDA;
    }
    ctx->own_stream = true;
  }
  ctx->b = params->b;
  ctx->P = params->P;
  ctx->kind = params->kind;
  ctx->keep_y = (params->flags & LRA_FLAG_KEEP_Y) != 0;
  const int64_t mn = std::min(m, n);
  ctx->nblk_max = params->k > 0 ? (params->k + ctx->b - 1) / ctx->b
                  : params->max_blocks > 0 ? params->max_blocks
                                           : (mn + 2 * ctx->b - 1) / (2 * ctx->b);
  ctx->lmax = ctx->nblk_max * ctx->b;

  OmegaSpec& os = ctx->os;
  os.kind = params->kind;
  os.n = n;
  os.b = params->b;
  os.zeta = params->zeta;
  os.k0 = (uint32_t)(params->seed & 0xFFFFFFFFull);
  os.k1 = (uint32_t)(params->seed >> 32);
  os.p = 0.0;
  os.thr = 0;
  os.inv_scale = 1.0;
  if (params->kind == LRA_OMEGA_SPARSE_SIGN) {
    os.inv_scale = 1.0 / sqrt((double)params->zeta);
    ctx->sparse = true;
    ctx->cap = params->zeta;
  } else if (params->kind == LRA_OMEGA_GAUSSIAN) {
    ctx->sparse = false;
  } else {
    os.p = params->p > 0.0 ? params->p : default_p(params->kind, n, params->zeta);
    os.thr = (uint64_t)floor(os.p * 4294967296.0);
    if (params->kind == LRA_OMEGA_SPARSE_SIGN_IID || params->kind == LRA_OMEGA_SPARSE_GAUSSIAN)
      os.inv_scale = 1.0 / sqrt(os.p);
    ctx->sparse = (double)n * os.p <= (double)SPARSE_MAX_NNZ_PER_COL;
    ctx->cap = (int)n;
  }
  ctx->sb_sparse = ctx->sparse && params->kind == LRA_OMEGA_STD_BERNOULLI;

  ctx->ldq = round_up(m, 2);
  ctx->ldb = round_up(std::max<int64_t>(ctx->lmax, 1), 2);
  ctx->lds = round_up(std::max(m, n), 2);
  ctx->ldf = round_up(std::max<int64_t>(ctx->lmax, 1), 2);
  ctx->ldod = round_up(n, 2);
  ctx->ws_elems = dgemm_ws_elems();
  const int b = ctx->b;
#define ALLOC(ptr, count)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = dalloc(ctx, &ctx->ptr, (count));                                      \
    if (e_ != cudaSuccess) {                                                               \
      lra_status r_ = fail(ctx, e_ == cudaErrorMemoryAllocation ? LRA_ERR_OOM : LRA_ERR_CUDA, \
                           "allocating %s: %s", #ptr, cudaGetErrorString(e_));             \
      free_all(ctx);                                                                       \
      delete ctx;                                                                          \
      cudaGetLastError();                                                                  \
      return r_;                                                                           \
    }                                                                                      \
  } while (0)
  ALLOC(Q, ctx->ldq * ctx->lmax);
  ALLOC(B, ctx->ldb * n);
  if (ctx->keep_y) ALLOC(Yk, ctx->ldq * ctx->lmax);
  ALLOC(S0, ctx->lds * b);
  ALLOC(Yb, ctx->lds * b);
  ALLOC(T1, ctx->lds * b);
  ALLOC(Tmp, ctx->lds * b);
  ALLOC(W, ctx->lds * b);
  ALLOC(G, ctx->lds * b);
  ALLOC(Wt, ctx->lds * b);
  ALLOC(F, ctx->ldf * b);
  ALLOC(BOm, ctx->ldf * b);
  ALLOC(z, m);
  ALLOC(zB, ctx->ldb);
  ALLOC(wvec, n);
  ALLOC(ws, ctx->ws_elems);
  ALLOC(gram, LRA_MAX_B * LRA_MAX_B);
  ALLOC(Rinv, LRA_MAX_B * LRA_MAX_B);
  ALLOC(dead, LRA_MAX_B);
  ALLOC(near, 2);
  ALLOC(colsq, std::max<int64_t>(n, LRA_MAX_B));
  ALLOC(colsum, std::max<int64_t>(n, LRA_MAX_B));
  ALLOC(scal, 8);
  ALLOC(flags, 4);
  ctx->tensor = (params->flags & LRA_FLAG_FP64_SIMT) == 0;
  ctx->graphs = (params->flags & LRA_FLAG_NO_GRAPHS) == 0;
  ctx->mixed = (params->flags & LRA_FLAG_MIXED) != 0;
  if (!dry) {
    // kernel attributes, before any stream capture
    cudaError_t e = gather_prepare();
    if (e == cudaSuccess && ctx->tensor) e = oz_prepare();
    if (e != cudaSuccess) {
      lra_status r = fail(ctx, LRA_ERR_CUDA, "kernel attributes: %s", cudaGetErrorString(e));
      free_all(ctx);
      delete ctx;
      return r;
    }
  }
  if (ctx->tensor) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 152;  // sizing without a device (dry run): the GB300's SM count
    }
    ctx->oz.ctas = sms > 0 ? sms : 1;
    ctx->oz.img_bytes = oz_img_bytes(std::max(m, n));
    ALLOC(rowE, m);
    ALLOC(colE, n);
    ALLOC(qrowE, m);
    ALLOC(qcolE, ctx->ldb);
    ALLOC(browE, ctx->ldb);
    ALLOC(bcolE, n);
    ALLOC(xrowE, ctx->lds);
    ALLOC(xcolE, LRA_MAX_B);
    ALLOC(oz.yE, LRA_MAX_B);
    ALLOC(oz.img, ctx->oz.img_bytes);
    ALLOC(oz.part, oz_part_elems(ctx->oz.ctas));
    ALLOC(oz.count, 1);
    if (!ctx->dry && cudaMemsetAsync(ctx->oz.count, 0, sizeof(int), ctx->st) != cudaSuccess) {
      const lra_status r_ = fail(ctx, LRA_ERR_CUDA, "cudaMemsetAsync of the arrival counter failed");
      cudaGetLastError();
      free_all(ctx);
      delete ctx;
      return r_;
    }
    // the statistics pass's partial sums, or the digit cut's (one per CTA)
    ALLOC(astat, std::max<int64_t>(a_stats_part_elems(m, n), 4 * (int64_t)ctx->oz.ctas));
    // A's digit images when the device has room (else every pass cuts A itself)
    if (!(params->flags & LRA_FLAG_NO_A_DIGITS)) {
      const int64_t b0 = oz_ximg_bytes(m, n), b1 = oz_ximg_bytes(n, m);
      const int64_t before = ctx->bytes;
      if (dalloc(ctx, &ctx->ximg[0], b0) != cudaSuccess ||
          dalloc(ctx, &ctx->ximg[1], b1) != cudaSuccess) {
        cudaGetLastError();
        dfree(ctx, ctx->ximg[0]);
        ctx->ximg[0] = ctx->ximg[1] = nullptr;
        ctx->bytes = before;
      }
    }
  }
  if (ctx->sparse) {
    ALLOC(om_counts, b);
    ALLOC(om_rows, (int64_t)b * ctx->cap);
    ALLOC(om_vals, (int64_t)b * ctx->cap);
  } else {
    ALLOC(om_dense, ctx->ldod * b);
  }
#undef ALLOC
  if (dry) {
    *out = ctx;
    return LRA_OK;
  }
  ctx->hp = pinned_arena().get();
  cudaError_t e = ctx->hp ? cudaSuccess : cudaErrorMemoryAllocation;
  if (e != cudaSuccess) {
    free_all(ctx);
    delete ctx;
    cudaGetLastError();
    return LRA_ERR_OOM;
  }
  if (params->flags & LRA_FLAG_PROFILE) {
    ctx->prof = true;
    for (int i = 0; i < lra_ctx::NEV && e == cudaSuccess; ++i) {
      e = cudaEventCreate(&ctx->ev0[i]);
      if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1[i]);
    }
    if (e != cudaSuccess) {
      free_all(ctx);
      delete ctx;
      return LRA_ERR_CUDA;
    }
  }
  // zB must start at zero: rows are written as blocks are appended.
  e = cudaMemsetAsync(ctx->zB, 0, ctx->ldb * sizeof(double), ctx->st);
  if (e != cudaSuccess) {
    free_all(ctx);
    delete ctx;
    return LRA_ERR_CUDA;
  }
  *out = ctx;
  return LRA_OK;
}

}  // namespace

lra_status lra_create(lra_ctx** out, int64_t m, int64_t n, const lra_params* params,
                      void* cuda_stream) {
  return create_ctx(out, m, n, params, cuda_stream, false);
}

int64_t lra_workspace_bytes(int64_t m, int64_t n, const lra_params* params) {
  lra_ctx* ctx = nullptr;
  const lra_status s = create_ctx(&ctx, m, n, params, nullptr, true);
  if (s != LRA_OK) return s;
  const int64_t bytes = ctx->bytes + (int64_t)sizeof(Pinned);
  delete ctx;
  return bytes;
}

int64_t lra_device_bytes(const lra_ctx* ctx) { return ctx ? ctx->bytes : -1; }

lra_status lra_selftest_waits(int* which) {
  if (which) *which = 0;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return LRA_ERR_CUDA;
  int w = 0;
  const cudaError_t e = wait_selftest(&w, st);
  cudaStreamDestroy(st);
  if (e != cudaSuccess) return LRA_ERR_CUDA;
  if (which) *which = w;
  return w ? LRA_ERR_TIMEOUT : LRA_OK;
}

void lra_destroy(lra_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  else cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
}

lra_status lra_farpca_run(lra_ctx* ctx, const lra_matrix* A) {
  if (!ctx) return LRA_ERR_INVALID_ARG;
  ctx->err.clear();
  TRY(check_matrix(ctx, A, true));
  return run(ctx, A->data, A->lda, A->dtype);
}

lra_status lra_svd(lra_ctx* ctx, lra_svd_t* out) {
  if (!ctx || !out) return LRA_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  ctx->err.clear();
  if (!ctx->run_ok) return fail(ctx, LRA_ERR_INVALID_ARG, "no completed lra_farpca_run");
  const int64_t l = ctx->rank, m = ctx->m, n = ctx->n;
  out->l = l;
  out->normA2 = ctx->normA2;
  if (l == 0) {
    out->E_r = ctx->normA2;
    return LRA_OK;
  }
  if (l > eig_max_l()) return fail(ctx, LRA_ERR_UNSUPPORTED, "l = %lld above %lld", (long long)l,
                                   (long long)eig_max_l());
  TRY(svd_alloc(ctx, l));
  auto& w = ctx->svd;
  cudaStream_t st = ctx->st;
  const bool tc = ctx->tensor;
  CK(transpose(ctx->B, ctx->ldb, l, n, w.Bt, n, st));
  if (tc) {
    CK(oz_rowcol_exponents(w.Bt, n, n, l, w.btrowE, w.btcolE, st));
    CK(oz_rowcol_exponents(ctx->Q, ctx->ldq, m, l, w.qrowE, nullptr, st));
  }
  // the l x l Gram B B^T = Bt^T Bt, 64 columns per product
  for (int64_t c0 = 0; c0 < l; c0 += 64) {
    const int64_t nc = std::min<int64_t>(64, l - c0);
    TRY(mm(ctx, true, l, nc, n, 1.0, w.Bt, n, tc ? w.btcolE : nullptr, w.Bt + c0 * n, n, 0.0,
           w.G + c0 * l, 1, l, tc ? w.btcolE + c0 : nullptr));
  }
  CK(eig_sym(w.G, l, (int)l, w.C0, w.C1, w.V, SVD_MAX_SWEEPS, SVD_JACOBI_TOL, w.bar, w.info, st));  // C1: snapshot
  int info[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(info, w.info, sizeof info, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (info[0] & FLAG_TIMEOUT) return fail(ctx, LRA_ERR_TIMEOUT, "eigensolver barrier wait gave up");
  CK(eig_sort(w.C0, (int)l, w.sigma, w.perm, w.vinv, w.V, w.Vs, w.W, st));
  // U = Q Vt, V = Bt Vt sigma^{-1}
  for (int64_t c0 = 0; c0 < l; c0 += 64) {
    const int64_t nc = std::min<int64_t>(64, l - c0);
    TRY(mm(ctx, false, m, nc, l, 1.0, ctx->Q, ctx->ldq, tc ? w.qrowE : nullptr, w.Vs + c0 * l, l,
           0.0, w.U + c0 * m, 1, m));
    TRY(mm(ctx, false, n, nc, l, 1.0, w.Bt, n, tc ? w.btrowE : nullptr, w.W + c0 * l, l, 0.0,
           w.Vout + c0 * n, 1, n));
  }
  std::vector<double> sig(l);
  CK(cudaMemcpyAsync(sig.data(), w.sigma, l * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  // post-processing truncation (Sec. 5.3): first r with E_r below the threshold
  double E = ctx->normA2;
  int64_t r = l;
  if (ctx->prm.k > 0) {
    r = std::min<int64_t>(ctx->prm.k, l);
    for (int64_t i = 0; i < r; ++i) E -= sig[i] * sig[i];
  } else {
    const double thr = ctx->prm.eps * ctx->prm.eps * ctx->normA2;
    for (int64_t i = 0; i < l; ++i) {
      E -= sig[i] * sig[i];
      if (E < thr) {
        r = i + 1;
        break;
      }
    }
  }
  out->status = info[2] ? LRA_OK : LRA_NOT_CONVERGED;
  out->sweeps = info[1];
  out->r = r;
  out->E_r = E;
  out->U = w.U;
  out->ldu = m;
  out->sigma = w.sigma;
  out->V = w.Vout;
  out->ldv = n;
  return LRA_OK;
}

lra_status lra_phase_times(lra_ctx* ctx, double* ms, int64_t* calls, int32_t nphases,
                           int32_t reset) {
  if (!ctx || nphases < 0 || nphases > LRA_NUM_PHASES) return LRA_ERR_INVALID_ARG;
  TRY(prof_flush(ctx));
  for (int i = 0; i < nphases; ++i) {
    if (ms) ms[i] = ctx->phase_ms[i];
    if (calls) calls[i] = ctx->phase_calls[i];
  }
  if (reset)
    for (int i = 0; i < LRA_NUM_PHASES; ++i) {
      ctx->phase_ms[i] = 0.0;
      ctx->phase_calls[i] = 0;
    }
  return LRA_OK;
}

lra_status lra_result(const lra_ctx* ctx, lra_result_t* out) {
  if (!ctx || !out) return LRA_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  out->status = ctx->status;
  out->rank = ctx->rank;
  out->blocks = ctx->blocks;
  out->E = ctx->E;
  out->normA2 = ctx->normA2;
  out->rel_err = ctx->normA2 > 0.0 ? sqrt(std::max(ctx->E, 0.0) / ctx->normA2) : 0.0;
  out->Q = ctx->Q;
  out->ldq = ctx->ldq;
  out->B = ctx->B;
  out->ldb = ctx->ldb;
  out->Y = ctx->keep_y ? ctx->Yk : nullptr;
  out->ldy = ctx->keep_y ? ctx->ldq : 0;
  return LRA_OK;
}

lra_status lra_sketch(lra_ctx* ctx, const lra_matrix* A, int64_t j0, int64_t nblk, double* Y,
                      int64_t ldy) {
  if (!ctx) return LRA_ERR_INVALID_ARG;
  ctx->err.clear();
  TRY(check_matrix(ctx, A, true));
  if (A->dtype == LRA_F32 && (!ctx->sparse || ctx->sb_sparse))
    return fail(ctx, LRA_ERR_UNSUPPORTED,
                "LRA_F32 sketches are implemented for the sparse (pure gather) kinds");
  if (j0 < 0 || nblk < 0 || j0 + nblk > (int64_t)UINT32_MAX)
    return fail(ctx, LRA_ERR_INVALID_ARG, "block range out of [0, 2^32)");
  if (nblk == 0) return LRA_OK;
  if (!Y || ldy < ctx->m) return fail(ctx, LRA_ERR_INVALID_ARG, "Y is NULL or ldy < m");
  const double* Ad = (const double*)A->data;
  const int b = ctx->b;
  if (!ctx->sparse) {
    TRY(a_exponents(ctx, Ad, A->lda));
    for (int64_t j = j0; j < j0 + nblk; ++j) {
      CK(omega_dense(ctx->os, j, 1, ctx->om_dense, ctx->ldod, ctx->st));
      TRY(dense(ctx, false, b, 1.0, Ad, A->lda, ctx->om_dense, ctx->ldod, 0.0, Y + (j - j0) * b * ldy,
                1, ldy));
    }
    return LRA_OK;
  }
  if (ctx->sb_sparse) {
    TRY(a_exponents(ctx, Ad, A->lda));
    TRY(compute_z(ctx, Ad, A->lda));
  }
  int64_t chunk = std::max<int64_t>(1, SKETCH_SCRATCH_ENTRIES / ((int64_t)b * ctx->cap));
  chunk = std::min(chunk, nblk);
  TRY(ensure_sketch_scratch(ctx, chunk * b, ctx->cap));
  CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int), ctx->st));
  for (int64_t j = j0; j < j0 + nblk; j += chunk) {
    const int64_t nb = std::min(chunk, j0 + nblk - j);
    CK(omega_sparse(ctx->os, j, nb, ctx->cap, ctx->sk_counts, ctx->sk_rows, ctx->sk_vals,
                    ctx->flags, ctx->st));
    CK(gather_sketch(A->data, A->dtype, A->lda, ctx->m, ctx->sk_counts, ctx->sk_rows, ctx->sk_vals,
                     ctx->cap,
                     nb * b, Y + (j - j0) * b * ldy, ldy, ctx->sb_sparse ? ctx->z : nullptr,
                     ctx->flags, ctx->st));
  }
  return LRA_OK;
}

lra_status lra_apply(lra_ctx* ctx, const lra_matrix* A, int32_t trans, const double* Y, int64_t ldy,
                     int64_t N, double* C, int64_t ldc) {
  if (!ctx) return LRA_ERR_INVALID_ARG;
  ctx->err.clear();
  TRY(check_matrix(ctx, A));
  const int64_t rows_y = trans ? ctx->m : ctx->n, rows_c = trans ? ctx->n : ctx->m;
  if (!Y || !C || N < 1 || N > LRA_MAX_B || ldy < rows_y || ldc < rows_c)
    return fail(ctx, LRA_ERR_INVALID_ARG, "bad Y / C / N / ld");
  const double* Ad = (const double*)A->data;
  CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int), ctx->st));
  if (ctx->tensor)
    CK(oz_rowcol_exponents(Ad, A->lda, ctx->m, ctx->n, trans ? nullptr : ctx->rowE,
                           trans ? ctx->colE : nullptr, ctx->st));
  TRY(dense(ctx, trans != 0, N, 1.0, Ad, A->lda, Y, ldy, 0.0, C, 1, ldc));
  CK(cudaMemcpyAsync(&ctx->hp->flags, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (ctx->hp->flags & FLAG_TIMEOUT) return fail(ctx, LRA_ERR_TIMEOUT, "a device wait timed out");
  return LRA_OK;
}

lra_status lra_copy_omega(lra_ctx* ctx, int64_t j, int64_t cap, int32_t* counts, int32_t* rows,
                          double* vals) {
  if (!ctx || !counts || !rows || !vals) return LRA_ERR_INVALID_ARG;
  ctx->err.clear();
  const int b = ctx->b;
  const int64_t n = ctx->n;
  if (j < 0 || j > (int64_t)UINT32_MAX) return fail(ctx, LRA_ERR_INVALID_ARG, "j out of range");
  if (ctx->kind == LRA_OMEGA_GAUSSIAN) {
    if (cap < n) return fail(ctx, LRA_ERR_INVALID_ARG, "cap must be >= n");
    CK(omega_dense(ctx->os, j, 1, ctx->om_dense, ctx->ldod, ctx->st));
    CK(cudaMemcpy2DAsync(vals, cap * sizeof(double), ctx->om_dense, ctx->ldod * sizeof(double),
                         n * sizeof(double), b, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int c = 0; c < b; ++c) {
      counts[c] = (int32_t)n;
      for (int64_t t = 0; t < n; ++t) rows[c * cap + t] = (int32_t)t;
    }
    return LRA_OK;
  }
  const int dcap = ctx->kind == LRA_OMEGA_SPARSE_SIGN ? ctx->prm.zeta : (int)n;
  if (cap < dcap) return fail(ctx, LRA_ERR_INVALID_ARG, "cap must be >= %d", dcap);
  TRY(ensure_sketch_scratch(ctx, b, dcap));
  CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int), ctx->st));
  CK(omega_sparse(ctx->os, j, 1, dcap, ctx->sk_counts, ctx->sk_rows, ctx->sk_vals, ctx->flags,
                  ctx->st));
  CK(cudaMemcpyAsync(counts, ctx->sk_counts, b * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpy2DAsync(rows, cap * sizeof(int32_t), ctx->sk_rows, dcap * sizeof(int32_t),
                       dcap * sizeof(int32_t), b, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpy2DAsync(vals, cap * sizeof(double), ctx->sk_vals, dcap * sizeof(double),
                       dcap * sizeof(double), b, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaMemcpyAsync(&ctx->hp->flags, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (ctx->hp->flags & FLAG_OMEGA_CAP)
    return fail(ctx, LRA_ERR_INVALID_ARG, "fixed-zeta draws exhausted");
  return LRA_OK;
}

namespace {

// A_host (m x n, ld lda_host, elements of type dtype) into device buffer dst (ld
// ctx->ldq elements) in NCOPY column chunks, one per copy stream (several copy
// engines at once), each after the work already on `after` (an event, or none).
// Returns with the chunks queued; ctx->cev[i] marks the end of chunk i.
lra_status copy_in(lra_ctx* ctx, const void* A_host, int dtype, int64_t lda_host, void* dst_buf,
                   cudaEvent_t after) {
  const int64_t m = ctx->m, n = ctx->n;
  const size_t es = dtype == LRA_F32 ? sizeof(float) : sizeof(double);
  char* dst = reinterpret_cast<char*>(dst_buf);
  const char* src = reinterpret_cast<const char*>(A_host);
  for (int i = 0; i < lra_ctx::NCOPY; ++i) {
    const int64_t c0 = i * n / lra_ctx::NCOPY, c1 = (i + 1) * n / lra_ctx::NCOPY;
    if (after) CK(cudaStreamWaitEvent(ctx->cst[i], after, 0));
    if (c1 > c0)
      CK(cudaMemcpy2DAsync(dst + c0 * ctx->ldq * es, ctx->ldq * es, src + c0 * lda_host * es,
                           lda_host * es, m * es, c1 - c0, cudaMemcpyHostToDevice, ctx->cst[i]));
    CK(cudaEventRecord(ctx->cev[i], ctx->cst[i]));
  }
  return LRA_OK;
}

// lra_farpca_host for either element type: A_host (m x n, ld lda_host) is copied
// in column chunks into a staging buffer of the context (ld = ldq elements of that
// type) and run there -- unless the previous call prefetched exactly that source,
// whose copy is then used.  next (may be NULL): a source whose copy into the other
// buffer starts before the run, on the copy streams, so that it overlaps it.
lra_status host_run(lra_ctx* ctx, const void* A_host, int dtype, int64_t lda_host, double* Q_host,
                    int64_t ldq_host, double* B_host, int64_t ldb_host, lra_result_t* out,
                    const void* next = nullptr) {
  if (!ctx || !A_host) return LRA_ERR_INVALID_ARG;
  ctx->err.clear();
  const int64_t m = ctx->m, n = ctx->n;
  if (lda_host < m) return fail(ctx, LRA_ERR_INVALID_ARG, "lda_host < m");
  if (Q_host && ldq_host < m) return fail(ctx, LRA_ERR_INVALID_ARG, "ldq_host < m");
  if (B_host && ldb_host < ctx->lmax) return fail(ctx, LRA_ERR_INVALID_ARG, "ldb_host < capacity");
  if (!ctx->A_host_copy) CK(dalloc(ctx, &ctx->A_host_copy, ctx->ldq * n));
  if (next && !ctx->A_host_copy2) CK(dalloc(ctx, &ctx->A_host_copy2, ctx->ldq * n));
  if (!ctx->cstart) {
    CK(cudaEventCreateWithFlags(&ctx->cstart, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->pref_ev, cudaEventDisableTiming));
    for (int i = 0; i < lra_ctx::NCOPY; ++i) {
      CK(cudaStreamCreateWithFlags(&ctx->cst[i], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&ctx->cev[i], cudaEventDisableTiming));
    }
  }
  double* buf[2] = {ctx->A_host_copy, ctx->A_host_copy2};
  const bool have = ctx->pref_valid && ctx->pref_host == A_host && ctx->pref_lda == lda_host &&
                    ctx->pref_dtype == dtype;
  int cur = 0;
  if (have) {
    // the prefetched copy: the run waits for it on the device
    cur = ctx->pref_buf;
    CK(cudaStreamWaitEvent(ctx->st, ctx->pref_ev, 0));
  } else {
    // another source: a prefetch in flight (into either buffer) must land first
    if (ctx->pref_valid) CK(cudaEventSynchronize(ctx->pref_ev));
    cur = ctx->pref_valid ? 1 - ctx->pref_buf : 0;
    if (!buf[cur]) cur = 0;
    CK(cudaEventRecord(ctx->cstart, ctx->st));
    TRY(copy_in(ctx, A_host, dtype, lda_host, buf[cur], ctx->cstart));
    for (int i = 0; i < lra_ctx::NCOPY; ++i) CK(cudaStreamWaitEvent(ctx->st, ctx->cev[i], 0));
  }
  ctx->pref_valid = false;
  if (next) {
    // the next source into the other buffer, behind this call's own copy on the
    // copy streams (the other buffer's last run ended with the previous call)
    const int nb = 1 - cur;
    TRY(copy_in(ctx, next, dtype, lda_host, buf[nb], nullptr));
    for (int i = 1; i < lra_ctx::NCOPY; ++i) CK(cudaStreamWaitEvent(ctx->cst[0], ctx->cev[i], 0));
    CK(cudaEventRecord(ctx->pref_ev, ctx->cst[0]));
    ctx->pref_host = next;
    ctx->pref_lda = lda_host;
    ctx->pref_dtype = dtype;
    ctx->pref_buf = nb;
    ctx->pref_valid = true;
  }
  lra_status s = run(ctx, buf[cur], ctx->ldq, dtype);
  if (s < 0) return s;
  if (Q_host && ctx->rank > 0)
    CK(cudaMemcpy2DAsync(Q_host, ldq_host * sizeof(double), ctx->Q, ctx->ldq * sizeof(double),
                         m * sizeof(double), ctx->rank, cudaMemcpyDeviceToHost, ctx->st));
  if (B_host && ctx->rank > 0)
    CK(cudaMemcpy2DAsync(B_host, ldb_host * sizeof(double), ctx->B, ctx->ldb * sizeof(double),
                         ctx->rank * sizeof(double), n, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (out) lra_result(ctx, out);
  return s;
}

}  // namespace

lra_status lra_farpca_host(lra_ctx* ctx, const double* A_host, int64_t lda_host, double* Q_host,
                           int64_t ldq_host, double* B_host, int64_t ldb_host, lra_result_t* out) {
  return host_run(ctx, A_host, LRA_F64, lda_host, Q_host, ldq_host, B_host, ldb_host, out);
}

lra_status lra_farpca_host_prefetch(lra_ctx* ctx, const double* A_host, int64_t lda_host,
                                    const double* A_next_host, double* Q_host, int64_t ldq_host,
                                    double* B_host, int64_t ldb_host, lra_result_t* out) {
  return host_run(ctx, A_host, LRA_F64, lda_host, Q_host, ldq_host, B_host, ldb_host, out, A_next_host);
}

lra_status lra_farpca_host_f32(lra_ctx* ctx, const float* A_host, int64_t lda_host, double* Q_host,
                               int64_t ldq_host, double* B_host, int64_t ldb_host,
                               lra_result_t* out) {
  return host_run(ctx, A_host, LRA_F32, lda_host, Q_host, ldq_host, B_host, ldb_host, out);
}

}  // extern "C"
