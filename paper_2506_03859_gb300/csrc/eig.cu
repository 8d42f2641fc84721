// The SVD that farPCA returns (arxiv 2506.03859, Alg. 1 / Alg. 2, the two
// eigendecompositions after the loop), in the QB form of the loop: with
// B = Q^T A (l x n), B B^T = Vt diag(lambda) Vt^T, sigma = sqrt(lambda) in
// descending order, U = Q Vt, V = B^T Vt diag(sigma)^{-1}.  This file holds the
// l x l symmetric eigendecomposition and the small kernels around it; the Gram
// B B^T and the lifts by Q and B^T run on the FP64-accurate tensor-core GEMM.
//
// Eigensolver: cyclic two-sided Jacobi (Jacobi 1846; the rotation of Golub and
// Van Loan, "Matrix Computations", Sec. 8.5) with the round-robin ordering, in
// which one round rotates l/2 disjoint index pairs at once and l - 1 rounds
// make a sweep that meets every pair once.  One cooperative launch runs all
// sweeps: a round is one grid-wide pass that applies the round's rotations to
// the 2 x 2 blocks of C (C <- J^T C J, in place: every element belongs to
// exactly one block of the round) and to the rows of the eigenvector matrix
// (V <- V J), then a grid barrier.  The round's pairs are cut into S slices and
// the work into S (S + 1) / 2 CTAs, one per pair of slices (ka <= kb), so that a
// CTA computes only the rotations of its two slices (FP64 square roots and
// divisions are the long part of a round on this GPU's narrow FP64 pipe).  The
// three entries each pair of the next round needs (c_pp, c_qq, c_pq) are
// written, by the threads that produce them, into a small double-buffered
// snapshot, so the rotations come from the same values in every CTA without
// re-reading C.  Each slice's rotations are counted once per sweep in a global
// counter (three slots in turn, so that one is read, one filled and one cleared
// in any sweep); a sweep whose count is zero ends the iteration, a decision
// every CTA reads after the same barrier.  A block whose two rotations are
// both the identity is left as it is.  A thread's first block and first
// eigenvector rows are loaded before the round's rotations are computed (their
// indices depend on the round alone), so those loads overlap the rotations.
// A pair is skipped when |c_pq| <= tol sqrt(|c_pp c_qq|): the relative
// criterion under which Jacobi keeps the small eigenvalues of a positive
// definite matrix to high relative accuracy (Demmel and Veselic, SIAM J. Matrix
// Anal. Appl. 13 (1992)).  The barrier's waits are bounded; a wait that gives
// up sets FLAG_TIMEOUT and every CTA returns.
#include <math.h>

#include <algorithm>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace lra {
namespace {

constexpr int EIG_NT = 256;
constexpr long long EIG_SPIN_LIMIT = 1ll << 22;  // polls (an L2 round trip and 32 ns each): ~3 s

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a cooperative launch (all CTAs resident).  bar[0]
// counts arrivals over the whole launch and is never reset: the k-th barrier
// (k = 0, 1, ...) is passed once it reaches nblocks (k + 1), so an arrival is
// one fire-and-forget reduction and the release needs no extra step by the last
// CTA (the count stays below 2^32 for any launch: nblocks * rounds).  Returns
// false when this CTA gave up waiting (and set FLAG_TIMEOUT in *info); the
// other CTAs then give up at their next wait, each after the same bounded spin.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned passed, int* info, int* s_ok,
                             long long limit = EIG_SPIN_LIMIT) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = nblocks * (passed + 1u);
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
    int ok = 1;
    long long it = 0;
    while ((int)(ld_acquire(bar) - target) < 0) {
      if (++it > limit) {
        atomicOr(info, FLAG_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Pair index of index x in round t (the inverse of round_pair).
__device__ __forceinline__ int pair_of(int x, int t, int lp) {
  if (x == 0) return 0;
  const int M = lp - 1;
  int i = (x - 1 - t) % M;
  if (i < 0) i += M;
  if (i == 0) return 0;
  return i < lp / 2 ? i : M - i;
}

// Pair k (0 <= k < lp/2) of round t (0 <= t < lp - 1) of the circle ordering:
// index 0 stays, indices 1 .. lp-1 sit on a ring of lp - 1 seats that turns by
// one seat per round; seat i faces seat lp-1-i, seat 0 faces index 0.
__device__ __forceinline__ void round_pair(int k, int t, int lp, int& p, int& q) {
  const int M = lp - 1;
  auto seat = [&](int i) {
    int v = i + t;
    if (v >= M) v -= M;
    return 1 + v;
  };
  int a, b;
  if (k == 0) {
    a = 0;
    b = seat(0);
  } else {
    a = seat(k);
    b = seat(M - k);
  }
  p = min(a, b);
  q = max(a, b);
}

struct Rot {
  double c, s, t;  // cos, sin, tan; s == 0 means no rotation
};

// The rotation J (J_pp = J_qq = c, J_pq = s, J_qp = -s) with (J^T C J)_pq = 0:
// t = tan = sgn(theta) / (|theta| + sqrt(theta^2 + 1)), theta = x / y with
// x = c_qq - c_pp, y = 2 c_pq, c = 1 / sqrt(1 + t^2), s = t c.  Multiplying by |y|
// gives t = sgn(x) y / (|x| + sqrt(x^2 + y^2)), one FP64 division fewer on the
// round's critical path (FP64 division and square root are long sequences on
// this GPU); the theta form is kept where x^2 + y^2 could overflow or
// underflow.  The skip test is evaluated beside the rotation, not before it.
__device__ __forceinline__ Rot jacobi_rot(double app, double aqq, double apq, double tol) {
  const bool skip = apq == 0.0 || fabs(apq) <= tol * sqrt(fabs(app) * fabs(aqq));
  const double x = aqq - app, y = 2.0 * apq;
  const double mx = fmax(fabs(x), fabs(y));
  double t;
  if (mx < 1e150 && mx > 1e-150) {
    t = copysign(1.0, x) * y / (fabs(x) + sqrt(fma(x, x, y * y)));
  } else {
    const double theta = x / y;
    t = fabs(theta) > 1e150 ? 0.5 / theta
                            : copysign(1.0, theta) / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
  }
  Rot r{1.0, 0.0, 0.0};
  if (skip) return r;
  const double c = rsqrt(fma(t, t, 1.0));
  r.c = c;
  r.s = t * c;
  r.t = t;
  return r;
}

struct EigArgs {
  double* C;      // lp x lp, ld lp (symmetric), updated in place
  double* snap;   // 2 x (lp/2) x 3: c_pp, c_qq, c_pq of each pair of a round
  double* V;      // lp x lp eigenvectors (columns), starts as I
  int l, lp, max_sweeps;
  int S, sz;      // pair slices of a round (S (S + 1) / 2 CTAs), pairs per slice
  double tol;
  unsigned* bar;  // arrival count, zero at launch
  int* rotcnt;    // 3 per-sweep rotation counters, zero at launch
  int* info;      // [0] flags, [1] sweeps, [2] converged, [3] 0
};

// An element (x, y) of C holding value v after round t: if x and y form a pair
// of the next round (or x == y belongs to one), record v in that pair's
// snapshot entry.
__device__ __forceinline__ void snap_put(double* nsnap, int x, int y, double v, int tn, int lp) {
  const int kx = pair_of(x, tn, lp);
  if (kx != pair_of(y, tn, lp)) return;
  int p, q;
  round_pair(kx, tn, lp, p, q);
  const int slot = x != y ? 2 : (x == p ? 0 : 1);
  nsnap[3 * kx + slot] = v;
}

// Block w of a CTA's 2 x 2 blocks: (i, j) = (w div nbk, w mod nbk) for two
// different slices, else i <= j within the slice with w = j (j + 1) / 2 + i.
__device__ __forceinline__ void block_of(int w, bool two, int nbk, int& i, int& j) {
  if (two) {
    i = w / nbk;
    j = w - i * nbk;
  } else {
    j = 0;
    while ((j + 1) * (j + 2) / 2 <= w) ++j;
    i = w - j * (j + 1) / 2;
  }
}

// The pairs of a round are cut into S slices of sz consecutive pair indices; CTA
// (ka, kb), ka <= kb, applies the 2 x 2 blocks (P, R) with P in slice ka and R
// in slice kb (P <= R), and rotates the eigenvector rows of slice ka in row
// chunk kb and of slice kb in row chunk ka (the rows split in S chunks).  It
// needs the rotations of its two slices only.  Every block and every (row,
// pair) belongs to exactly one CTA.
__global__ void __launch_bounds__(EIG_NT) k_jacobi(EigArgs a) {
  extern __shared__ double sm[];
  const int lp = a.lp, nb2 = lp / 2, M = lp - 1, sz = a.sz;
  double* rc = sm;              // cos of the CTA's 2 sz pairs (slice ka, then slice kb)
  double* rs = rc + 2 * sz;     // sin
  double* rt = rs + 2 * sz;     // tan
  int2* pq = reinterpret_cast<int2*>(rt + 2 * sz);
  __shared__ int s_ok;
  int kb = 0;
  while ((kb + 1) * (kb + 2) / 2 <= (int)blockIdx.x) ++kb;
  const int ka = (int)blockIdx.x - kb * (kb + 1) / 2;
  const int a0 = ka * sz, na = max(0, min(sz, nb2 - a0));
  const int b0 = kb * sz, nbk = max(0, min(sz, nb2 - b0));
  const int rch = (a.l + a.S - 1) / a.S;
  double* C = a.C;
  int sweep = 0, converged = 0;
  int64_t g = 0;  // rounds done
  for (; sweep < a.max_sweeps && !converged; ++sweep) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(a.rotcnt + (sweep + 1) % 3, 0);
    for (int t = 0; t < M; ++t, ++g) {
      const double* csnap = a.snap + (g & 1) * 3 * nb2;
      double* nsnap = a.snap + ((g + 1) & 1) * 3 * nb2;
      const int tn = t + 1 == M ? 0 : t + 1;
      // The thread's first 2 x 2 block and first eigenvector rows are loaded
      // before the rotations are known: their indices depend on the round alone,
      // so the loads overlap the rotation arithmetic.
      const int nblk = ka < kb ? na * nbk : na * (na + 1) / 2;
      double pz[4] = {0.0, 0.0, 0.0, 0.0}, pv[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
      if ((int)threadIdx.x < nblk) {
        int i, j, p, q;
        block_of((int)threadIdx.x, ka < kb, nbk, i, j);
        round_pair(a0 + i, t, lp, p, q);
        if (ka == kb && i == j) {
          pz[0] = __ldcg(C + (int64_t)p * lp + p);
          pz[1] = __ldcg(C + (int64_t)q * lp + q);
          pz[2] = __ldcg(C + (int64_t)q * lp + p);
        } else {
          int r, s2i;
          round_pair((ka < kb ? b0 : a0) + j, t, lp, r, s2i);
          pz[0] = __ldcg(C + (int64_t)r * lp + p);
          pz[1] = __ldcg(C + (int64_t)s2i * lp + p);
          pz[2] = __ldcg(C + (int64_t)r * lp + q);
          pz[3] = __ldcg(C + (int64_t)s2i * lp + q);
        }
      }
      for (int part = 0; part < (ka < kb ? 2 : 1); ++part) {
        const int np = part ? nbk : na, c0 = (part ? ka : kb) * rch;
        const int rows = max(0, min(a.l, c0 + rch) - c0);
        if ((int)threadIdx.x < np * rows) {
          const int u = (int)threadIdx.x / rows, i = c0 + ((int)threadIdx.x - u * rows);
          int p, q;
          round_pair((part ? b0 : a0) + u, t, lp, p, q);
          pv[part][0] = __ldcg(a.V + (int64_t)p * lp + i);
          pv[part][1] = __ldcg(a.V + (int64_t)q * lp + i);
        }
      }
      // the rotations of the CTA's two slices: from C itself before the first
      // round, else from the snapshot the previous round wrote
      int rotated = 0;
      for (int slot = threadIdx.x; slot < 2 * sz; slot += EIG_NT) {
        const int h = slot / sz, u = slot % sz;
        const int k = (h ? b0 : a0) + u;
        if (u < (h ? nbk : na)) {
          int p, q;
          round_pair(k, t, lp, p, q);
          double app, aqq, apq;
          if (g == 0) {
            app = __ldcg(C + (int64_t)p * lp + p);
            aqq = __ldcg(C + (int64_t)q * lp + q);
            apq = __ldcg(C + (int64_t)q * lp + p);
          } else {
            app = __ldcg(csnap + 3 * k);
            aqq = __ldcg(csnap + 3 * k + 1);
            apq = __ldcg(csnap + 3 * k + 2);
          }
          const Rot r = jacobi_rot(app, aqq, apq, a.tol);
          rc[slot] = r.c;
          rs[slot] = r.s;
          rt[slot] = r.t;
          pq[slot] = make_int2(p, q);
          // each slice's rotations are counted once, by its diagonal CTA
          rotated += (h == 0 && ka == kb && r.s != 0.0) ? 1 : 0;
        }
      }
      const int cnt = __syncthreads_count(rotated);
      if (cnt && threadIdx.x == 0) atomicAdd(a.rotcnt + sweep % 3, cnt);
      // 2 x 2 blocks (P, R): P in slice ka (slot i), R in slice kb (slot sz + j)
      for (int w = threadIdx.x; w < nblk; w += EIG_NT) {
        const bool first = w == (int)threadIdx.x;
        int i, j;
        block_of(w, ka < kb, nbk, i, j);
        const int sP = i, sR = ka < kb ? sz + j : j;
        const int p = pq[sP].x, q = pq[sP].y;
        const double c1 = rc[sP], s1 = rs[sP];
        if (ka == kb && i == j) {
          double npp = first ? pz[0] : __ldcg(C + (int64_t)p * lp + p);
          double nqq = first ? pz[1] : __ldcg(C + (int64_t)q * lp + q);
          double npq = first ? pz[2] : __ldcg(C + (int64_t)q * lp + p);
          if (s1 != 0.0) {
            const double apq = npq;
            npp = fma(-rt[sP], apq, npp);
            nqq = fma(rt[sP], apq, nqq);
            npq = 0.0;
            __stcg(C + (int64_t)p * lp + p, npp);
            __stcg(C + (int64_t)q * lp + q, nqq);
            __stcg(C + (int64_t)q * lp + p, npq);
            __stcg(C + (int64_t)p * lp + q, npq);
          }
          snap_put(nsnap, p, p, npp, tn, lp);
          snap_put(nsnap, q, q, nqq, tn, lp);
          snap_put(nsnap, p, q, npq, tn, lp);
        } else {
          const int r = pq[sR].x, s2i = pq[sR].y;
          const double c2 = rc[sR], s2 = rs[sR];
          double z00, z01, z10, z11;
          if (first) {
            z00 = pz[0];
            z01 = pz[1];
            z10 = pz[2];
            z11 = pz[3];
          } else {
            z00 = __ldcg(C + (int64_t)r * lp + p);
            z01 = __ldcg(C + (int64_t)s2i * lp + p);
            z10 = __ldcg(C + (int64_t)r * lp + q);
            z11 = __ldcg(C + (int64_t)s2i * lp + q);
          }
          if (s1 != 0.0 || s2 != 0.0) {
            // Y = J_P^T X, then X' = Y J_R
            const double y00 = c1 * z00 - s1 * z10, y01 = c1 * z01 - s1 * z11;
            const double y10 = s1 * z00 + c1 * z10, y11 = s1 * z01 + c1 * z11;
            z00 = c2 * y00 - s2 * y01;
            z01 = s2 * y00 + c2 * y01;
            z10 = c2 * y10 - s2 * y11;
            z11 = s2 * y10 + c2 * y11;
            __stcg(C + (int64_t)r * lp + p, z00);
            __stcg(C + (int64_t)s2i * lp + p, z01);
            __stcg(C + (int64_t)r * lp + q, z10);
            __stcg(C + (int64_t)s2i * lp + q, z11);
            __stcg(C + (int64_t)p * lp + r, z00);
            __stcg(C + (int64_t)p * lp + s2i, z01);
            __stcg(C + (int64_t)q * lp + r, z10);
            __stcg(C + (int64_t)q * lp + s2i, z11);
          }
          snap_put(nsnap, p, r, z00, tn, lp);
          snap_put(nsnap, p, s2i, z01, tn, lp);
          snap_put(nsnap, q, r, z10, tn, lp);
          snap_put(nsnap, q, s2i, z11, tn, lp);
        }
      }
      // eigenvector rows: (slice ka, row chunk kb) and, off the diagonal, (slice kb, chunk ka)
      for (int part = 0; part < (ka < kb ? 2 : 1); ++part) {
        const int np = part ? nbk : na, base = part ? sz : 0;
        const int c0 = (part ? ka : kb) * rch, c1r = min(a.l, c0 + rch);
        const int rows = max(0, c1r - c0);
        for (int w = threadIdx.x; w < np * rows; w += EIG_NT) {
          const int u = w / rows, i = c0 + (w - u * rows);
          const double s1 = rs[base + u];
          if (s1 != 0.0) {
            const double c1 = rc[base + u];
            double* vp = a.V + (int64_t)pq[base + u].x * lp + i;
            double* vq = a.V + (int64_t)pq[base + u].y * lp + i;
            const bool first = w == (int)threadIdx.x;
            const double xp = first ? pv[part][0] : __ldcg(vp), xq = first ? pv[part][1] : __ldcg(vq);
            __stcg(vp, c1 * xp - s1 * xq);
            __stcg(vq, s1 * xp + c1 * xq);
          }
        }
      }
      if (!grid_barrier(a.bar, gridDim.x, (unsigned)g, a.info, &s_ok)) return;
    }
    converged = atomicAdd(a.rotcnt + sweep % 3, 0) == 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.info[1] = sweep;
    a.info[2] = converged;
    a.info[3] = 0;
  }
}

// C0[i, j] = G[min(i,j), max(i,j)] for i, j < l (the upper triangle of the
// Gram, ld ldg), zero in the padding; V = I.
__global__ void k_eig_init(const double* __restrict__ G, int64_t ldg, int l, int lp,
                           double* __restrict__ C0, double* __restrict__ V) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)lp * lp) return;
  const int j = (int)(e / lp), i = (int)(e - (int64_t)j * lp);
  double c = 0.0;
  if (i < l && j < l) c = i <= j ? G[i + (int64_t)j * ldg] : G[j + (int64_t)i * ldg];
  C0[e] = c;
  V[e] = i == j ? 1.0 : 0.0;
}

// Descending order of the eigenvalues lambda_i = C[i, i] (ties by index):
// sigma[rank] = sqrt(max(lambda, 0)), perm[rank] = i, vinv[rank] = 1 / ||V[:, i]||.
// Every rotation leaves c^2 + s^2 within a rounding error of 1, but for small
// angles that error leans to one side, and thousands of rotations per column
// move the column norms by up to ~1e-13; renormalising removes that drift
// (the pairwise orthogonality error stays a random walk).
__global__ void k_eig_rank(const double* __restrict__ C, const double* __restrict__ V, int l, int lp,
                           double* __restrict__ sigma, int* __restrict__ perm,
                           double* __restrict__ vinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= l) return;
  const double li = C[(int64_t)i * lp + i];
  int rank = 0;
  for (int j = 0; j < l; ++j) {
    const double lj = C[(int64_t)j * lp + j];
    rank += (lj > li) || (lj == li && j < i);
  }
  double ss = 0.0;
  const double* v = V + (int64_t)i * lp;
  for (int j = 0; j < l; ++j) ss = fma(v[j], v[j], ss);
  sigma[rank] = sqrt(fmax(li, 0.0));
  perm[rank] = i;
  vinv[rank] = 1.0 / sqrt(ss);
}

// Vs[:, k] = V[0:l, perm[k]] vinv[k] and W[:, k] = Vs[:, k] / sigma[k] (0 if
// sigma[k] == 0), both l x l, ld l.
__global__ void k_eig_gather(const double* __restrict__ V, int l, int lp, const int* __restrict__ perm,
                             const double* __restrict__ vinv, const double* __restrict__ sigma,
                             double* __restrict__ Vs, double* __restrict__ W) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)l * l) return;
  const int k = (int)(e / l), i = (int)(e - (int64_t)k * l);
  const double v = V[(int64_t)perm[k] * lp + i] * vinv[k];
  const double s = sigma[k];
  Vs[e] = v;
  W[e] = s > 0.0 ? v / s : 0.0;
}

// Bt (n x l, ld ldt) = transpose of B (l x n, ld ldb); 32 x 32 tiles.
__global__ void k_transpose(const double* __restrict__ B, int64_t ldb, int64_t l, int64_t n,
                            double* __restrict__ Bt, int64_t ldt) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + threadIdx.x, c = c0 + y;
    if (r < l && c < n) tile[y][threadIdx.x] = B[r + c * ldb];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t c = c0 + threadIdx.x, r = r0 + y;
    if (r < l && c < n) Bt[c + r * ldt] = tile[threadIdx.x][y];
  }
}

// The two kinds of bounded device wait, each against a condition that never
// comes true: an mbarrier that expects one arrival nobody makes, and the grid
// barrier of a two-CTA group launched with one CTA.  Both must give up after
// their limit and report FLAG_TIMEOUT (info[0] bit 0: the mbarrier wait, bit 1:
// the grid barrier), leaving the context usable.  One CTA of 32 threads.
__global__ void k_wait_selftest(unsigned* bar, int* info) {
  __shared__ uint64_t mb;
  __shared__ int s_ok;
  if (threadIdx.x == 0) tc::mbar_init(&mb, 1);
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(&mb, 0u, 1L << 14)) atomicOr(info, 1);
  if (!grid_barrier(bar, 2u, 0u, info + 1, &s_ok, 1ll << 14) && threadIdx.x == 0) atomicOr(info, 2);
}

}  // namespace

int64_t eig_padded(int64_t l) { return l + (l & 1); }

int64_t eig_max_l() {
  // the per-CTA rotation table (32 bytes a pair) must fit in shared memory
  return 2 * ((200 * 1024) / 32);
}

cudaError_t eig_sym(const double* G, int64_t ldg, int l, double* C0, double* snap, double* V,
                    int max_sweeps, double tol, unsigned* bar, int* info, cudaStream_t st) {
  if (l < 1 || l > eig_max_l()) return cudaErrorInvalidValue;
  const int lp = (int)eig_padded(l);
  const int64_t elems = (int64_t)lp * lp;
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(info, 0, 4 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_eig_init<<<(unsigned)((elems + 255) / 256), 256, 0, st>>>(G, ldg, l, lp, C0, V);
  e = launched();
  if (e != cudaSuccess) return e;
  const int nb2 = lp / 2;
  static std::atomic<bool> attr{false};  // concurrent first calls set it twice, harmlessly
  if (!attr.load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr.store(true, std::memory_order_release);
  }
  int dev = 0, sms = 0, occ = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // S pair slices -> S (S + 1) / 2 CTAs, about one per SM (and co-resident)
  int S = 1;
  while (S < nb2 && (S + 1) * (S + 2) / 2 <= sms) ++S;
  const int sz = (nb2 + S - 1) / S;
  const size_t smem = (size_t)2 * sz * 32;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_jacobi, EIG_NT, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1 || S * (S + 1) / 2 > occ * sms) return cudaErrorInvalidConfiguration;
  const int64_t grid = (int64_t)S * (S + 1) / 2;
  e = cudaMemsetAsync(bar + 2, 0, 3 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  EigArgs a{C0, snap, V, l, lp, max_sweeps, S, sz, tol, bar, reinterpret_cast<int*>(bar + 2), info};
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)k_jacobi, dim3((unsigned)grid), dim3(EIG_NT), args,
                                  smem, st);
  if (e != cudaSuccess) return e;
  return launched();
}

cudaError_t eig_sort(const double* C, int l, double* sigma, int* perm, double* vinv, const double* V,
                     double* Vs, double* W, cudaStream_t st) {
  const int lp = (int)eig_padded(l);
  k_eig_rank<<<(l + 127) / 128, 128, 0, st>>>(C, V, l, lp, sigma, perm, vinv);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  const int64_t elems = (int64_t)l * l;
  k_eig_gather<<<(unsigned)((elems + 255) / 256), 256, 0, st>>>(V, l, lp, perm, vinv, sigma, Vs, W);
  return launched();
}

cudaError_t transpose(const double* B, int64_t ldb, int64_t l, int64_t n, double* Bt, int64_t ldt,
                      cudaStream_t st) {
  if (l <= 0 || n <= 0) return cudaSuccess;
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((l + 31) / 32));
  k_transpose<<<grid, dim3(32, 8), 0, st>>>(B, ldb, l, n, Bt, ldt);
  return launched();
}

// Runs k_wait_selftest on its own buffers; *which = the waits that gave up
// (bit 0: mbarrier, bit 1: grid barrier).
cudaError_t wait_selftest(int* which, cudaStream_t st) {
  *which = 0;
  int* buf = nullptr;  // [0] bar, [1] bits, [2] the grid barrier's flags
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), 4 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(buf, 0, 4 * sizeof(int), st);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, st>>>(reinterpret_cast<unsigned*>(buf), buf + 1);
    e = cudaGetLastError();
  }
  int host[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, buf, sizeof(host), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(buf, st);
  if (e == cudaSuccess) {
    e = cudaStreamSynchronize(st);
    *which = host[1] & 3;
    if (!(host[2] & FLAG_TIMEOUT)) *which &= ~2;
  }
  return e;
}

}  // namespace lra
