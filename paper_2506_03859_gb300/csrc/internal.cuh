// Internal declarations shared by the library's translation units.
// Every kernel launch goes through a host wrapper declared here; wrappers bump
// the process-wide launch counter and return the launch's cudaError_t.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/lra.h"

namespace lra {

extern std::atomic<uint64_t> g_launches;

inline cudaError_t launched() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

// Device-side error bits (a single int in device memory, read once per block).
enum : int {
  FLAG_BREAKDOWN = 1,     // a Cholesky pivot failed the breakdown test
  FLAG_OMEGA_CAP = 2,     // fixed-zeta generator ran out of draws
  FLAG_TIMEOUT = 4,       // a bounded device wait gave up
};

// Philox stream tags (counter word 3); see philox.cuh.
enum : uint32_t { TAG_SPARSE_SIGN = 1, TAG_MASK = 2, TAG_GAUSS = 3, TAG_FILL = 4 };

// ---------------------------------------------------------------- omega.cu
struct OmegaSpec {
  int kind;            // lra_omega_kind
  int64_t n;           // rows of Omega
  int b;               // columns per block
  int zeta;            // fixed-zeta kind
  double p;            // Bernoulli probability (i.i.d. kinds)
  uint64_t thr;        // floor(p * 2^32)
  double inv_scale;    // 1/sqrt(zeta) or 1/sqrt(p)
  uint32_t k0, k1;     // Philox key
};

// Sparse structure of Omega for blocks j0 .. j0 + nblk - 1 (nblk * b columns):
// counts[g], rows[g * cap + t], vals[g * cap + t].  Fixed-zeta kind or i.i.d.
// mask kinds (values: 1 for the Bernoulli / standardized Bernoulli kinds).
cudaError_t omega_sparse(const OmegaSpec& s, int64_t j0, int64_t nblk, int cap, int* counts,
                         int* rows, double* vals, int* flags, cudaStream_t st);
// Dense Omega (n x (nblk*b), ld ldo): Gaussian; standardized Bernoulli as the
// shifted Bernoulli matrix B - p (Alg. 2 with the scale dropped); other kinds
// as their definition.
cudaError_t omega_dense(const OmegaSpec& s, int64_t j0, int64_t nblk, double* Om, int64_t ldo,
                        cudaStream_t st);
// Columns c < b of X (rows x b, ld ldx) with dead[c] != 0 become +-1/sqrt(rows)
// from the TAG_FILL stream, counter (r, j, c + 64 step): the directions that
// replace the dependent columns of a power-step panel.
cudaError_t fill_dead(double* X, int64_t ldx, int64_t rows, int b, const int* dead, uint32_t k0,
                      uint32_t k1, int64_t j, int step, cudaStream_t st);

// ---------------------------------------------------------------- sketch.cu
// Y[i, g] = sum_t vals[g*cap+t] * X[i, rows[g*cap+t]] - (shift ? shift[i] : 0)
// for i < rows_x, g < ncols; X column-major with ld ldx.  A bounded device wait
// that gives up sets FLAG_TIMEOUT in *flags.
// Kernel attributes (dynamic shared memory) set once per process, before any
// stream capture; the prepare functions are idempotent.
cudaError_t gather_prepare();
cudaError_t gather_sketch(const void* X, int dtype, int64_t ldx, int64_t rows_x, const int* counts,
                          const int* rows, const double* vals, int cap, int64_t ncols, double* Y,
                          int64_t ldy, const double* shift, int* flags, cudaStream_t st);

// ---------------------------------------------------------------- dgemm_simt.cu
// C[p, c] = alpha * sum_k opX[p, k] Y[k, c] + beta * C[p, c], p < P, c < N <= 64.
// trans: opX[p, k] = X[k + p*ldx] (X is K x P); else opX[p, k] = X[p + k*ldx].
// C element (p, c) at C[p*csp + c*csc].  beta == 0 never reads C.
// ws: split-K workspace of ws_elems doubles.
struct GemmOut {
  double* C;
  int64_t csp, csc;
};
cudaError_t dgemm(bool trans, int64_t P, int64_t N, int64_t K, double alpha, const double* X,
                  int64_t ldx, const double* Y, int64_t ldy, double beta, GemmOut out, double* ws,
                  int64_t ws_elems, cudaStream_t st);
int64_t dgemm_ws_elems();

// ---------------------------------------------------------------- ozgemm.cu
// FP64-accurate C = alpha op(X) Y + beta C on the tcgen05 tensor cores (error-free
// bf16 slicing).  xE: biased max exponent of each row of op(X) (P entries).
struct OzWorkspace {
  int* count;        // arrival counter of the fused Gram + Cholesky (zero between launches)
  int* yE;           // 64 ints
  uint8_t* img;      // pre-sliced Y, img_bytes
  int64_t img_bytes;
  double* part;      // partial tiles, oz_part_elems(ctas)
  int ctas;          // CTAs of the persistent grid (one per SM)
};
int64_t oz_img_bytes(int64_t K);
cudaError_t oz_prepare();
int64_t oz_part_elems(int ctas);
// Largest K the tensor engine accepts (its exact int64 sums stay in range).
int64_t oz_max_k();
// yE_known: biased max exponents of Y's columns when the caller has them.
// chol: the product is a b x b Gram (C column-major with ld b); factor it in the
// same launch as the Gram's fixup (k_oz_fixup_chol), as chol_inv would.
// skip: NULL, or every launch of the product does nothing while *skip != 0 (not
// with chol; Y's exponents known or K <= 4096).
struct CholJob {
  double* Rinv;
  int* dead;   // NULL: breakdown ends the factorisation; else skip mode (chol_inv)
  int* count;  // the workspace's arrival counter
  double tau;
  int* near;   // NULL, or the near-identity flag of chol_inv
};
cudaError_t ozgemm(bool trans, int64_t P, int64_t N, int64_t K, double alpha, const double* X,
                   int64_t ldx, const int* xE, const double* Y, int64_t ldy, double beta, GemmOut out,
                   const OzWorkspace& w, int* flags, cudaStream_t st, const int* yE_known = nullptr,
                   const CholJob* chol = nullptr, const int* skip = nullptr);
// The digit image of op(X) (P x K): every (128-row tile, 16-deep stage) as seven
// f16 digit planes, cut once and reused by ozgemm_img.  xE as for ozgemm.
int64_t oz_ximg_bytes(int64_t P, int64_t K);
// sqpart (when given): one partial sum of squares of op(X)'s entries per CTA of
// the cut, oz_cut_ctas(P, K, ctas) of them; summed in order they give ||X||_F^2.
int oz_cut_ctas(int64_t P, int64_t K, int ctas);
cudaError_t oz_cut_x(bool trans, int64_t P, int64_t K, const void* X, int dtype, int64_t ldx,
                     const int* xE, uint8_t* ximg, int ctas, cudaStream_t st,
                     double* sqpart = nullptr);
// low: the reduced form (digits 0..3 of both operands; ~2^-30 of max|x| max|y|).
// ydig1: every column of Y is a multiple of a single power of two (its entries
// 0 and +-2^k, e.g. a +-1/2 test matrix), so Y's digits beyond the first are zero
// and only the pairs (s, 0) are multiplied: the same result, exactly, from a
// quarter of the tensor work and one Y digit plane per stage.
cudaError_t ozgemm_img(int64_t P, int64_t N, int64_t K, double alpha, const uint8_t* ximg,
                       const int* xE, const double* Y, int64_t ldy, double beta, GemmOut out,
                       const OzWorkspace& w, int* flags, cudaStream_t st, bool low = false,
                       bool ydig1 = false);
// rowE[r] / colE[c] = largest biased exponent in row r / column c of X (either may
// be NULL).  accumulate_rows: rowE[r] = max(rowE[r], ...) instead of overwriting.
// skip: NULL, or the launches do nothing while *skip != 0 (only where no
// exponent array is zeroed first: rows <= 4096 for colE, cols < 256 and no
// accumulation for rowE).
cudaError_t oz_rowcol_exponents(const double* X, int64_t ld, int64_t rows, int64_t cols,
                                int* rowE, int* colE, cudaStream_t st, bool accumulate_rows = false,
                                const int* skip = nullptr);

// ---------------------------------------------------------------- orth.cu
// Per-column sums of squares and/or sums of X (rows x cols, ld): one CTA per column.
cudaError_t col_sums(const double* X, int64_t ld, int64_t rows, int64_t cols, double* sumsq,
                     double* sum, cudaStream_t st);
// One pass over A: colsq[c] = ||A[:, c]||^2 (summed over 512-row blocks through
// part, a_stats_part_elems(m, n) doubles), colE / rowE = largest biased exponent
// of each column / row.  Deterministic.
int64_t a_stats_part_elems(int64_t m, int64_t n);
// part == NULL: the exponents only (colsq not written).
cudaError_t a_stats(const void* A, int dtype, int64_t lda, int64_t m, int64_t n, double* part,
                    double* colsq, int* colE, int* rowE, cudaStream_t st);
// out[0] = sum of v[0..count) in a fixed order (one CTA).
cudaError_t total(const double* v, int64_t count, double* out, cudaStream_t st);
// Cholesky S = R^T R (S: b x b, ld b), R^{-1} into Rinv (b x b, ld b); on a failed
// pivot (d_c not > tau * S_cc or not finite) sets FLAG_BREAKDOWN in *flags.
// With dead != NULL a failed pivot instead marks its column dependent (dead[c] = 1,
// every entry of dead[0..b) written): the column takes no part in the other
// columns' factor, and row and column c of Rinv are zero.
// near (when given): set to 1 when every entry of S - I is within 2^-40 (X R^{-1}
// may then be taken as rinv_near_identity computes it), else 0.
cudaError_t chol_inv(const double* S, int b, double tau, double* Rinv, int* flags, cudaStream_t st,
                     int* dead = nullptr, int* near = nullptr);
// out (rows x b, ld ldo) = X + X (Rinv - I) with the correction in FP32, when
// *near != 0 (see chol_inv); otherwise the launch does nothing.  b <= 64; out and
// X do not overlap.
cudaError_t rinv_near_identity(const double* X, int64_t ldx, int64_t rows, int b, const double* Rinv,
                               const int* near, double* out, int64_t ldo, cudaStream_t st);
// The second projection of CGS2, Y -= Q F (Q: rows x l, ld ldq; F: l x b, ld ldf;
// Y: rows x b, ld ldy), in FP32 when every |F[k, c]| is below the bound that keeps
// the FP32 sum's error within 2^-53 of Y's column scale (yE: biased exponents of
// Y's column maxima); *taken = 1 then, else 0 and Y is left as it was.  b <= 64.
cudaError_t project_fp32(const double* Q, int64_t ldq, int64_t rows, int64_t l, const double* F,
                         int64_t ldf, int b, const int* yE, double* Y, int64_t ldy, int* taken,
                         cudaStream_t st);
// B[row0 + c, r] = Wt[r, c] (Wt: n x b, ld ldw); zB[row0 + c] = p * colsum[c] if zB.
cudaError_t append_rows(const double* Wt, int64_t ldw, int64_t n, int b, double* B, int64_t ldb,
                        int64_t row0, const double* colsum, double p, double* zB, cudaStream_t st);
// X[i, c] = v for all i < rows, c < cols.
cudaError_t fill(double* X, int64_t ld, int64_t rows, int64_t cols, double v, cudaStream_t st);

// ---------------------------------------------------------------- eig.cu
// Cyclic Jacobi eigendecomposition of a symmetric l x l matrix given by the upper
// triangle of G (ld ldg): one cooperative launch.  C, V: eig_padded(l)^2 doubles
// each (the eigenvalues end on C's diagonal, the eigenvectors in V's columns);
// snap: 3 eig_padded(l) doubles; bar: 5 words (zeroed here); info: 4 ints ([0] flags,
// FLAG_TIMEOUT if a barrier wait gave up; [1] sweeps; [2] converged; [3] 0).
int64_t eig_padded(int64_t l);
int64_t eig_max_l();
// Bounded-wait self-test (k_wait_selftest): *which = the waits that gave up.
cudaError_t wait_selftest(int* which, cudaStream_t st);
cudaError_t eig_sym(const double* G, int64_t ldg, int l, double* C, double* snap, double* V,
                    int max_sweeps, double tol, unsigned* bar, int* info, cudaStream_t st);
// sigma (l, descending) = sqrt of the eigenvalues on C's diagonal; Vs = V's
// columns in that order, renormalised (l x l, ld l); W = Vs diag(sigma)^{-1}
// (0 where sigma = 0).  perm, vinv: l entries of scratch.
cudaError_t eig_sort(const double* C, int l, double* sigma, int* perm, double* vinv, const double* V,
                     double* Vs, double* W, cudaStream_t st);
// Bt (n x l, ld ldt) = B^T for B l x n (ld ldb).
cudaError_t transpose(const double* B, int64_t ldb, int64_t l, int64_t n, double* Bt, int64_t ldt,
                      cudaStream_t st);

}  // namespace lra
