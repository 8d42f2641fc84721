/*
 * lra.h -- fixed-precision randomized low-rank approximation on one GB300 GPU.
 *
 * The library runs the blocked farPCA loop (arxiv 2506.03859, Alg. 1; Alg. 2
 * for the standardized Bernoulli test matrix) with the paper's cheap test
 * matrices Omega (Def. 2.1-2.4) generated on the device from Philox4x32-10
 * counters.  Given a dense A (m x n) it builds, block of b columns by block,
 * an orthonormal Q (m x l) and B = Q^T A (l x n) until the Frobenius error
 * indicator E = ||A||_F^2 - ||B||_F^2 = ||A - QB||_F^2 (Sec. 2.1) drops below
 * eps^2 ||A||_F^2 (the relative test of Sec. 5.2), or a fixed rank is reached.
 *
 * Conventions for every entry point:
 *  - Matrices are column-major (element (i, j) at ptr[i + j * ld]), FP64
 *    unless an entry point states that it takes FP32 (LRA_F32) data.
 *  - "device" pointers are CUDA device memory of the current device; "host"
 *    pointers are ordinary (ideally pinned) host memory.  The library never
 *    frees memory it did not allocate.
 *  - All device work is ordered on the stream given to lra_create.
 *  - Return values: LRA_OK (0) or a positive status describing a run that
 *    ended early but left valid results; negative values are errors, after
 *    which lra_last_error(ctx) holds a message and outputs of the failing call
 *    are undefined.  A NULL ctx or NULL required pointer gives
 *    LRA_ERR_INVALID_ARG.
 *  - A context is not thread-safe: one host thread at a time per context.
 *    Different contexts may be created and used from different threads at once
 *    (the serving runtime does so); a server and a batch handle their own
 *    locking as stated at their entry points.
 *
 * Beyond the loop itself: the SVD the method returns and its truncation
 * (lra_svd), FP32 input (lra_farpca_run, lra_farpca_host_f32), a serving
 * runtime for streams of requests (lra_server_*) and a batched form for many
 * small problems in one graph launch (lra_batch_*).
 */
#ifndef LRA_H
#define LRA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LRA_VERSION 1
#define LRA_MAX_B 64      /* largest block size b */
#define LRA_MAX_P 8       /* largest number of power steps P */
#define LRA_MAX_ZETA 256  /* largest nonzeros per column, fixed-zeta sparse sign */

typedef enum {
  LRA_OK = 0,
  LRA_NOT_CONVERGED = 1,   /* block cap reached before E < eps^2 ||A||_F^2     */
  LRA_BREAKDOWN = 2,       /* a new block was numerically rank deficient: the
                              Cholesky pivot of its Gram matrix was not above
                              1e-13 times the diagonal entry; results are those
                              of the blocks before it                            */
  LRA_ERR_INVALID_ARG = -1,
  LRA_ERR_OOM = -2,
  LRA_ERR_CUDA = -3,
  LRA_ERR_TIMEOUT = -4,
  LRA_ERR_UNSUPPORTED = -5
} lra_status;

/* Test-matrix kinds (arxiv 2506.03859 Sec. 2.2). */
typedef enum {
  LRA_OMEGA_GAUSSIAN = 0,        /* standard Gaussian (farPCA, Alg. 1)                       */
  LRA_OMEGA_STD_BERNOULLI = 1,   /* standardized Bernoulli, Def. 2.3 (farPCASB, Alg. 2):
                                    sketch = A B_j - z, z = A (p 1), scale dropped          */
  LRA_OMEGA_SPARSE_SIGN = 2,     /* sparse sign, zeta distinct nonzeros +-1/sqrt(zeta) per
                                    column (the fixed-nonzero form after Def. 2.2)         */
  LRA_OMEGA_SPARSE_SIGN_IID = 3, /* sparse sign, i.i.d. form of Def. 2.2, +-1/sqrt(p)       */
  LRA_OMEGA_SPARSE_GAUSSIAN = 4, /* sparse Gaussian, Def. 2.4, B o G / sqrt(p)              */
  LRA_OMEGA_BERNOULLI = 5        /* Bernoulli matrix, Def. 2.1 (farPCAB of Sec. 5)          */
} lra_omega_kind;

typedef enum { LRA_F64 = 0, LRA_F32 = 1 } lra_dtype;

/* Flags for lra_params.flags. */
#define LRA_FLAG_KEEP_Y 1u  /* keep every block's pre-projection sketch Y_j (the
                               paper's cumulative Y of Alg. 1); costs m x l_max FP64 */
#define LRA_FLAG_PROFILE 2u /* time each phase of lra_farpca_run with CUDA events on
                               the context's stream (read with lra_phase_times)   */
#define LRA_FLAG_FP64_SIMT 4u /* run the full passes over A as FP64 FMAs on the CUDA
                               cores instead of the FP64-accurate tensor-core GEMM
                               (error-free 8-bit digit split); an order of
                               magnitude slower on GB300                           */
#define LRA_FLAG_NO_A_DIGITS 8u /* tensor-core engine: do not keep A's digit images.
                               By default lra_create also allocates two images of A
                               cut into seven f16 digits (row- and column-scaled,
                               14 bytes per element each, 28 m n bytes in all) when
                               the device has room; lra_farpca_run cuts A once into
                               them (phase LRA_PHASE_CUT) and every full pass then
                               streams the digits instead of cutting A again.  With
                               this flag, or when the images do not fit, each pass
                               cuts A on the fly (same results, bit for bit).     */
#define LRA_FLAG_NO_GRAPHS 16u /* launch every kernel of lra_farpca_run directly.  By
                               default the fixed kernel sequence of each block (and
                               of the set-up after ||A||_F^2) is captured once into a
                               CUDA graph, cached per block index and per A pointer,
                               and replayed; results are the same bit for bit.     */
#define LRA_FLAG_MIXED 32u /* mixed precision form (tensor-core engine with A's digit
                               images): the sketch and power-step passes (dense
                               Omega sketch, W_j, the extra power steps, Y_j) use
                               the top four of the seven digits of A and of their
                               right operand, ~2^-30 of max|x| max|y| per product;
                               B_j = Q_j^T A, the projections, Gram, Cholesky and
                               the indicator stay FP64-accurate, so E is exact for
                               the basis found.  Without the images the flag has
                               no effect.                                          */
#define LRA_FLAG_POOL 64u  /* allocate the context's device memory from the device's
                              stream-ordered pool on its stream (cudaMallocAsync),
                              so that creating and destroying contexts next to
                              running ones synchronises nothing but their own
                              stream; the serving runtime uses it               */

/* Phases of one block, for lra_phase_times. */
typedef enum {
  LRA_PHASE_OMEGA = 0,      /* Omega_j generation (Philox)                         */
  LRA_PHASE_SKETCH = 1,     /* S0 = A Omega_j                                      */
  LRA_PHASE_DENSE = 2,      /* one full pass over A: A^T X or A X (power steps,
                               Y_j = A G, B_j^T = A^T Q_j)                         */
  LRA_PHASE_DEFLATE = 3,    /* B Omega_j, B G and B^T F (deflation)                */
  LRA_PHASE_PROJECT = 4,    /* Q^T Y and Y - Q F, twice                            */
  LRA_PHASE_ORTH = 5,       /* Gram, Cholesky, triangular apply, twice             */
  LRA_PHASE_INDICATOR = 6,  /* ||A||_F^2, ||B_j||_F^2, append of B_j               */
  LRA_PHASE_CUT = 7,        /* A cut into its digit images (once per run; see
                               LRA_FLAG_NO_A_DIGITS)                              */
  LRA_NUM_PHASES = 8
} lra_phase;

/* A borrowed, read-only dense matrix. */
typedef struct {
  int64_t m, n;       /* rows, columns (>= 1)                                     */
  int64_t lda;        /* leading dimension in elements, >= m                      */
  int32_t dtype;      /* lra_dtype: LRA_F64; LRA_F32 where an entry point says so
                         (elsewhere LRA_ERR_UNSUPPORTED)                          */
  int32_t reserved;   /* must be 0                                                */
  const void* data;   /* device, column-major; must stay valid while a call runs  */
} lra_matrix;

/* Arguments of the problem statement (Alg. 1 / Alg. 2 REQUIRE lines). */
typedef struct {
  double eps;          /* relative Frobenius tolerance, > 0 in fixed-precision mode   */
  int64_t k;           /* fixed-rank mode: run ceil(k/b) blocks; 0 = fixed precision   */
  int32_t b;           /* block size, 1..min(m, n, LRA_MAX_B)                          */
  int32_t P;           /* power steps, 0..LRA_MAX_P                                    */
  int32_t kind;        /* lra_omega_kind                                               */
  int32_t zeta;        /* fixed-zeta sparse sign: nonzeros per column, 1..min(n,
                          LRA_MAX_ZETA); sparse Gaussian with p == 0: p = zeta / n     */
  double p;            /* Bernoulli probability of the i.i.d. kinds, in (0, 1);
                          0 selects Sec. 5.1's p1 = max(1e-3, ln n / n) for the
                          standardized Bernoulli kind, p2 = max(1e-3, 10/n) otherwise  */
  uint64_t seed;       /* Philox key: Omega_j depends only on (seed, j, kind, n, b)    */
  int32_t max_blocks;  /* block cap; 0 = ceil(min(m, n) / (2b)) (Sec. 5.2)             */
  uint32_t flags;      /* LRA_FLAG_* bits                                              */
} lra_params;

/* State after lra_farpca_run.  Device pointers are owned by the context and
   stay valid until the next run on it or lra_destroy. */
typedef struct {
  int32_t status;        /* lra_status of the last run                          */
  int32_t reserved;
  int64_t rank;          /* l = blocks * b                                      */
  int64_t blocks;
  double E;              /* indicator after the last accepted block             */
  double normA2;         /* ||A||_F^2                                           */
  double rel_err;        /* sqrt(max(E, 0) / normA2), 0 when normA2 == 0        */
  const double* Q;       /* device, m x rank, column-major, ld = ldq            */
  int64_t ldq;
  const double* B;       /* device, rank x n, column-major, ld = ldb            */
  int64_t ldb;
  const double* Y;       /* device, m x rank pre-projection sketches, or NULL   */
  int64_t ldy;
} lra_result_t;

typedef struct lra_ctx lra_ctx;

/* Create a context for m x n inputs: validates *params, allocates the device
   workspace for the largest rank the run can reach (l_max = block cap * b), and
   binds `cuda_stream` (a cudaStream_t).  With NULL the context creates and owns
   a blocking stream, which is ordered with the legacy default stream as NULL
   would be (the legacy stream itself cannot be captured into CUDA graphs).
   Errors: LRA_ERR_INVALID_ARG, LRA_ERR_OOM, LRA_ERR_CUDA.  *out is NULL on error. */
lra_status lra_create(lra_ctx** out, int64_t m, int64_t n, const lra_params* params,
                      void* cuda_stream);

/* Free the context and everything it allocated.  NULL is ignored. */
void lra_destroy(lra_ctx* ctx);

/* Largest rank a run of this context can return (l_max); -1 for NULL. */
int64_t lra_capacity(const lra_ctx* ctx);

/* Sketch pass (Alg. 1 G_j / Alg. 2 steps 4-7): Y = A [Omega_j0 ... Omega_{j0+nblk-1}]
   with the context's kind, seed and b; for the standardized Bernoulli kind each
   block is A B_j - z, z = A (p 1) (Sec. 3.1).  A must be m x n as at create.
   Y: device, m x (nblk * b), column-major, ld = ldy >= m, caller-owned.
   nblk = 0 is a no-op.  A may be LRA_F32 for the kinds whose sketch is a pure
   gather (sparse sign, sparse Gaussian, Bernoulli; entries converted exactly,
   FP64 sums).  Errors: LRA_ERR_INVALID_ARG, LRA_ERR_UNSUPPORTED, LRA_ERR_CUDA. */
lra_status lra_sketch(lra_ctx* ctx, const lra_matrix* A, int64_t j0, int64_t nblk,
                      double* Y, int64_t ldy);

/* One full pass over A with the context's dense engine -- the contraction of
   Alg. 1's A G_j and A^T Y_j: C = op(A) Y, op(A) = A^T when trans != 0, else A.
   Y: device, (trans ? m : n) x N, ld ldy; C: device, (trans ? n : m) x N, ld ldc;
   1 <= N <= LRA_MAX_B; caller-owned.  FP64 result; computed on the tensor cores
   by error-free bf16 slicing (error comparable to an FP64 GEMM) unless the
   context was created with LRA_FLAG_FP64_SIMT.  Errors: LRA_ERR_INVALID_ARG,
   LRA_ERR_CUDA, LRA_ERR_TIMEOUT. */
lra_status lra_apply(lra_ctx* ctx, const lra_matrix* A, int32_t trans, const double* Y, int64_t ldy,
                     int64_t N, double* C, int64_t ldc);

/* Run the blocked farPCA loop on A (device, m x n as at create) until
   E < eps^2 ||A||_F^2 (LRA_OK), the block cap (LRA_NOT_CONVERGED), a rank-deficient
   block (LRA_BREAKDOWN) or, with k > 0, ceil(k/b) blocks (LRA_OK).
   ||A||_F = 0 gives rank 0 and LRA_OK; a non-finite ||A||_F^2 gives
   LRA_ERR_INVALID_ARG.  Synchronises the stream once per block for the stop test.
   A may be LRA_F32 (FP32 data of the 20000 x 10000 kind in Sec. 5's setting):
   its entries are converted exactly to FP64 where they are read (the pass for
   ||A||_F^2, the digit cut, the sparse gather), so the run computes the same
   bits as on the FP64 conversion of A while reading half the bytes; this needs
   the tensor engine with digit images (LRA_ERR_UNSUPPORTED with
   LRA_FLAG_FP64_SIMT or LRA_FLAG_NO_A_DIGITS). */
lra_status lra_farpca_run(lra_ctx* ctx, const lra_matrix* A);

/* Copy the state of the last run into *out (no device work). */
lra_status lra_result(const lra_ctx* ctx, lra_result_t* out);

/* The SVD A ~ U diag(sigma) V^T that the method returns (Alg. 1 / Alg. 2, the
   eigendecompositions after the loop, in the loop's QB form: with B = Q^T A,
   B B^T = Vt diag(sigma^2) Vt^T, U = Q Vt, V = B^T Vt diag(sigma)^{-1}), and the
   post-processing truncation of Sec. 5.3.  Device pointers are owned by the
   context and stay valid until the next lra_svd, lra_farpca_run or
   lra_destroy. */
typedef struct {
  int32_t status;        /* LRA_OK; LRA_NOT_CONVERGED if the eigensolver reached
                            its sweep cap (results are then its last iterate)  */
  int32_t sweeps;        /* Jacobi sweeps taken                                 */
  int64_t l;             /* rank of the run's approximation: columns of U, V    */
  int64_t r;             /* truncated rank: the smallest r with
                            ||A||_F^2 - sum_{i<=r} sigma_i^2 < eps^2 ||A||_F^2
                            (accumulated in this order); l if none; min(k, l)
                            in fixed-rank mode                                   */
  double E_r;            /* ||A||_F^2 - sum_{i<=r} sigma_i^2                   */
  double normA2;         /* ||A||_F^2 of the run                                */
  const double* U;       /* device, m x l, column-major, ld = ldu               */
  int64_t ldu;
  const double* sigma;   /* device, l singular values, descending               */
  const double* V;       /* device, n x l, column-major, ld = ldv; a column whose
                            sigma is 0 is 0                                     */
  int64_t ldv;
} lra_svd_t;

/* Extract the SVD of the last run's Q B (see lra_svd_t).  The l x l Gram B B^T
   and the products Q Vt, B^T Vt sigma^{-1} run on the context's GEMM engine;
   the eigendecomposition is a cyclic Jacobi iteration on the device (one
   cooperative launch, at most 40 sweeps).  Allocates, on the first call that
   needs them, about (3 l^2 + 2 (l + 1)^2 + (m + 2n) l) doubles, grown when a
   later run reaches a larger l.  Synchronises the stream.  l = 0 gives r = 0,
   E_r = normA2 and NULL pointers.  Errors: LRA_ERR_INVALID_ARG (NULL argument,
   or the last run failed), LRA_ERR_UNSUPPORTED (l above 12800), LRA_ERR_OOM,
   LRA_ERR_CUDA, LRA_ERR_TIMEOUT (a bounded device wait gave up). */
lra_status lra_svd(lra_ctx* ctx, lra_svd_t* out);

/* End-to-end form with host buffers: copy A_host (m x n, ld lda_host) to a
   device buffer owned by the context (allocated on the first call), run
   lra_farpca_run, and copy Q into Q_host (m x rank, ld ldq_host >= m) and B
   into B_host (rank x n, ld ldb_host >= lra_capacity); both must hold
   lra_capacity(ctx) columns / rows.  Q_host or B_host may be NULL to skip that
   copy.  Returns the run's status; *out (if not NULL) receives lra_result. */
lra_status lra_farpca_host(lra_ctx* ctx, const double* A_host, int64_t lda_host,
                           double* Q_host, int64_t ldq_host, double* B_host,
                           int64_t ldb_host, lra_result_t* out);

/* lra_farpca_host for FP32 host data (A_host: m x n floats, ld lda_host); the
   run is lra_farpca_run's LRA_F32 form.  Q_host, B_host as for lra_farpca_host. */
lra_status lra_farpca_host_f32(lra_ctx* ctx, const float* A_host, int64_t lda_host,
                               double* Q_host, int64_t ldq_host, double* B_host,
                               int64_t ldb_host, lra_result_t* out);

/* lra_farpca_host for a stream of host matrices: solves A_host as
   lra_farpca_host does and, when A_next_host is not NULL, starts copying
   A_next_host (the same m x n shape and ld lda_host) into a second device buffer
   owned by the context before this solve begins, on the context's copy streams,
   so that the copy overlaps the solve.  A later call whose A_host is that same
   pointer with the same lda uses the copy instead of copying again; any other
   call first waits for it to land.  The caller keeps A_next_host's memory valid
   and unchanged until the call that solves it (or lra_destroy) returns.  Not in
   the paper (its timings start with A in memory); it exists so that a caller
   who solves many host-resident matrices pays the host-to-device copy of each
   while the previous one is being solved.  Errors: as lra_farpca_host. */
lra_status lra_farpca_host_prefetch(lra_ctx* ctx, const double* A_host, int64_t lda_host,
                                    const double* A_next_host, double* Q_host, int64_t ldq_host,
                                    double* B_host, int64_t ldb_host, lra_result_t* out);

/* Omega_j as generated on the device, copied to host buffers (for bit-exact
   comparison).  counts[b]: nonzeros of each column; rows[c * cap + t] and
   vals[c * cap + t], t < counts[c]: row index and value of column c's t-th entry,
   in generation order (draw order for the fixed-zeta kind, increasing row for
   the others; every row for the Gaussian kind).  For the standardized Bernoulli
   kind the entries are those of the Bernoulli matrix B_j (value 1).  cap must be
   >= zeta (fixed-zeta kind) or >= n (other kinds).  Synchronises the stream.
   Errors: LRA_ERR_INVALID_ARG, LRA_ERR_CUDA. */
lra_status lra_copy_omega(lra_ctx* ctx, int64_t j, int64_t cap, int32_t* counts,
                          int32_t* rows, double* vals);

/* Accumulated device time (ms, CUDA events) and number of timed calls of each
   phase since creation or the last reset, for a context created with
   LRA_FLAG_PROFILE (zeros otherwise).  ms and calls are host arrays of nphases
   (<= LRA_NUM_PHASES) entries; reset != 0 clears the counters after reading. */
lra_status lra_phase_times(lra_ctx* ctx, double* ms, int64_t* calls, int32_t nphases, int32_t reset);

/* Bytes of the device array that lra_sketch_noalloc uses as its only scratch. */
#define LRA_NOALLOC_SCRATCH_BYTES (8 << 20)

/* The sparse sketch of lra_sketch, Y = A [Omega_j0 ... Omega_{j0+nblk-1}], without
   any device allocation and without a context.  The paper has no counterpart:
   this entry point exists for callers that cannot allocate device memory while
   they run -- a service that reserves its whole memory budget at start-up, a
   host framework whose own allocator owns the device memory, or code that
   cannot afford the synchronisation a cudaMalloc may cause.  Its scratch (the
   generated Omega) is one file-scope device array of LRA_NOALLOC_SCRATCH_BYTES
   that every GPU loading the library keeps until the process exits.
   A, params (b, kind, zeta, p, seed; the other fields are ignored), j0, nblk,
   Y and ldy mean what they mean for lra_create / lra_sketch; cuda_stream is a
   cudaStream_t (NULL = legacy default stream).  Kinds: LRA_OMEGA_SPARSE_SIGN,
   LRA_OMEGA_SPARSE_SIGN_IID, LRA_OMEGA_SPARSE_GAUSSIAN, LRA_OMEGA_BERNOULLI;
   the others need a context (LRA_ERR_UNSUPPORTED).  Limit: one block's Omega,
   b * (4 + 12 cap) bytes with cap = zeta (fixed-zeta kind) or n (the i.i.d.
   kinds), must fit in the array minus 768 bytes, else LRA_ERR_INVALID_ARG;
   longer block ranges are processed in chunks.
   Every call looks up the array's device address in the current device's
   context (cudaGetSymbolAddress); the first call on a device also loads the
   library's device code there, so make that first call before any stream
   capture starts.  All calls share the array and leave the last call's
   contents in it: calls that can overlap on the GPU (other streams, other host
   threads) race on it, so issue them in order on one stream.  The call copies
   its error word to the host and synchronises its stream before returning.
   Errors: LRA_ERR_INVALID_ARG, LRA_ERR_UNSUPPORTED, LRA_ERR_CUDA, and
   LRA_ERR_TIMEOUT when a bounded device wait of the gather gave up (Y is then
   incomplete; the device stays usable). */
lra_status lra_sketch_noalloc(const lra_matrix* A, const lra_params* params, int64_t j0,
                              int64_t nblk, double* Y, int64_t ldy, void* cuda_stream);

/* Device bytes lra_create would allocate for these arguments (the same sizing,
   nothing allocated; the lazily grown buffers of lra_sketch, lra_svd and
   lra_farpca_host are not included), or a negative lra_status for invalid
   arguments.  The admission test of the serving runtime. */
int64_t lra_workspace_bytes(int64_t m, int64_t n, const lra_params* params);

/* Device bytes the context has allocated so far; -1 for NULL. */
int64_t lra_device_bytes(const lra_ctx* ctx);

/* Diagnostic: runs the library's two kinds of bounded device wait (an
   mbarrier wait as in the tensor-core GEMM, the grid barrier of the
   eigensolver) against conditions that never come true, each with a short
   limit (2^14 polls).  Every wait of the library ends this way when its
   limit runs out: the kernel records FLAG_TIMEOUT and returns, the call
   reports LRA_ERR_TIMEOUT, and the device stays usable.  Returns
   LRA_ERR_TIMEOUT when a wait gave up (the expected outcome: both), LRA_OK if
   none did, LRA_ERR_CUDA on a launch or copy error; *which (may be NULL) gets
   bit 0 for the mbarrier wait and bit 1 for the grid barrier.  Runs on its
   own stream and synchronises it. */
lra_status lra_selftest_waits(int* which);

/* ---- Serving runtime: a stream of independent requests on one GPU --------
   Each request is a fixed-precision (or fixed-rank) farPCA run on its own
   matrix.  Requests are admitted in arrival order when a worker slot is free
   and their workspace (lra_workspace_bytes) fits in the device-memory budget
   next to the running ones; each runs in its own context on its worker's
   stream, so the block steps of concurrent requests interleave on the GPU.
   The per-request state (A, Q, B, E, the block counter, the Philox key) stays
   on the device; a request's Omega depends only on its own seed, so its result
   is the same bits alone or in any mix. */
typedef struct lra_server lra_server;

typedef struct {
  int64_t hbm_budget;  /* device bytes the admitted requests may hold at once;
                          0 = 90% of the free device memory at creation       */
  int32_t slots;       /* requests run at once (worker threads), 1..64        */
  uint32_t flags;      /* LRA_FLAG_* added to every request's parameters
                          (LRA_FLAG_POOL is always added)                     */
} lra_server_params;

typedef struct {
  uint64_t id;         /* caller's tag, returned in the completion            */
  lra_matrix A;        /* device (LRA_F64 or LRA_F32), borrowed until the
                          request completes                                   */
  lra_params params;
  int32_t keep;        /* != 0: keep the context for the caller (its results via
                          lra_result / lra_svd; release with
                          lra_server_release), else free it on completion     */
  int32_t reserved;
} lra_request;

typedef struct {
  uint64_t id;
  int32_t status;      /* lra_status of the run, or of a failed create        */
  int32_t reserved;
  int64_t rank;
  double rel_err;
  double t_submit;     /* seconds on the server's clock (lra_server_clock)    */
  double t_admit;      /* admitted (first come, first served)                 */
  double t_start;      /* its context created                                 */
  double t_done;       /* run finished                                        */
  int64_t bytes;       /* device bytes the request held                       */
  lra_ctx* ctx;        /* the context when keep != 0 (else NULL)              */
} lra_completion;

/* Create a server and start its worker threads.  Errors: LRA_ERR_INVALID_ARG,
   LRA_ERR_CUDA. */
lra_status lra_server_create(lra_server** out, const lra_server_params* params);

/* Queue a request (returns at once).  LRA_ERR_INVALID_ARG for bad arguments,
   LRA_ERR_UNSUPPORTED when its workspace alone exceeds the budget. */
lra_status lra_server_submit(lra_server* srv, const lra_request* req);

/* Move up to max completions, oldest first, into out; returns their number.
   wait != 0 blocks until at least one is available or nothing is pending. */
int64_t lra_server_poll(lra_server* srv, lra_completion* out, int64_t max, int32_t wait);

/* Requests submitted and not yet completed. */
int64_t lra_server_pending(const lra_server* srv);

/* Free a kept request's context and return its bytes to the budget. */
lra_status lra_server_release(lra_server* srv, lra_ctx* ctx);

/* Seconds since the server was created (steady clock). */
double lra_server_clock(const lra_server* srv);

/* Wait for every pending request, stop the workers, free what they hold
   (including kept contexts not released).  NULL is ignored. */
void lra_server_destroy(lra_server* srv);

/* ---- Batched form: many independent problems, one graph launch -----------
   Fixed-precision farPCA (QB form, fixed-zeta sparse sign Omega) on each of
   `count` FP32 matrices, advanced together one block per step by a CUDA graph
   that repeats the block step on the device while a problem is active.  FP32
   data and passes; Gram sums, Cholesky factors, ||A||_F^2 and the indicator in
   FP64; the basis by shifted Cholesky QR3.  A problem's Omega_j depends only on
   its seed, so its result does not depend on the rest of the batch. */
typedef struct lra_batch lra_batch;

typedef struct {
  int64_t m, n, lda;   /* FP32 matrix, device, column-major, borrowed while the
                          batch exists; b <= min(m, n), zeta <= n              */
  const float* A;
  double eps;          /* relative tolerance, > 0                             */
  uint64_t seed;       /* Philox key of its Omega                             */
} lra_batch_item;

typedef struct {
  int32_t b;           /* block size: 8, 16 or 32                             */
  int32_t P;           /* power steps: 0 or 1                                 */
  int32_t zeta;        /* nonzeros per Omega column, 1..16                    */
  int32_t max_blocks;  /* per-problem block cap; 0 = ceil(min(m, n) / (2b))   */
  uint32_t flags;      /* LRA_FLAG_NO_GRAPHS: launch each step from the host
                          (reading after each step whether to go on) instead
                          of the graph; other bits must be 0                  */
} lra_batch_params;

typedef struct {
  int32_t status;      /* LRA_OK, LRA_NOT_CONVERGED, LRA_BREAKDOWN, or
                          LRA_ERR_INVALID_ARG for a non-finite A             */
  int32_t reserved;
  int64_t rank;
  double E, normA2, rel_err;
  const float* Q;      /* device, m x rank, ld = ldq (owned by the batch)     */
  int64_t ldq;
  const float* Bt;     /* device, n x rank = B^T, ld = ldbt                   */
  int64_t ldbt;
} lra_batch_result_t;

/* Validate the problems, allocate their workspaces (lra_batch_device_bytes)
   and build the graph.  Errors: LRA_ERR_INVALID_ARG, LRA_ERR_OOM, LRA_ERR_CUDA. */
lra_status lra_batch_create(lra_batch** out, const lra_batch_item* items, int64_t count,
                            const lra_batch_params* params, void* cuda_stream);
/* Run every problem to its stop test (two set-up kernels and one graph launch);
   synchronises the stream. */
lra_status lra_batch_run(lra_batch* batch);
/* State of problem i (in the order given to lra_batch_create) after the run. */
lra_status lra_batch_result(const lra_batch* batch, int64_t i, lra_batch_result_t* out);
/* Block steps the last run took (the largest rank / b); -1 for NULL. */
int64_t lra_batch_steps(const lra_batch* batch);
/* Device bytes of the batch's workspaces; -1 for NULL. */
int64_t lra_batch_device_bytes(const lra_batch* batch);
void lra_batch_destroy(lra_batch* batch);

/* Tile shapes of the batched products, per shape class: tn[c] columns per thread
   of the X^T Y products (A^T X, Q^T X, Q_j^T A; 64 threads, tiles of 64 tn[c]
   columns) for problems with n < 256 (c = 0), < 640 (1), the rest (2); nn[c] rows
   per thread of the row products (A G, X - Q F; tiles of 64 nn[c] rows) for
   m < 384, < 1200, the rest.  Each 1, 2 or 4; the default is 2 everywhere.  The
   tiling changes how the work is cut, not what any thread sums nor the order of
   its sums: results are the same bits under every tiling.  Not in the paper (its
   MATLAB code runs one matrix at a time). */
typedef struct {
  int32_t tn[3];
  int32_t nn[3];
} lra_batch_tiling;

/* Use tiling t from the next lra_batch_run on (rebuilds the tile lists and the
   graph; results of earlier runs are no longer readable).  Errors:
   LRA_ERR_INVALID_ARG (NULL, or an entry not 1, 2 or 4), LRA_ERR_CUDA. */
lra_status lra_batch_set_tiling(lra_batch* batch, const lra_batch_tiling* t);
lra_status lra_batch_get_tiling(const lra_batch* batch, lra_batch_tiling* t);
/* The autotuner: coordinate descent over the knobs of the shape classes the
   batch holds (each tried at 1, 2 and 4 with the others fixed, in the order
   tn[0..2], nn[0..2]), every candidate timed by `reps` (>= 1) runs of the whole
   batch on its stream (CUDA events; the minimum counts).  Leaves the fastest
   tiling in place and returns it in *best and its time (ms per run) in *best_ms;
   *base_ms gets the time of the tiling in place at the call (either pointer may
   be NULL).  Synchronises the stream; results of earlier runs are no longer
   readable.  Errors: LRA_ERR_INVALID_ARG, LRA_ERR_CUDA. */
lra_status lra_batch_tune(lra_batch* batch, int32_t reps, lra_batch_tiling* best, double* best_ms,
                          double* base_ms);

/* Message for the last error on ctx ("" if none); never NULL. */
const char* lra_last_error(const lra_ctx* ctx);

/* Name of a status code. */
const char* lra_status_string(int32_t status);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t lra_kernel_launches(void);

/* LRA_VERSION of the built library. */
int32_t lra_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LRA_H */
