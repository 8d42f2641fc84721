// Host-side plan of a batch of the batched form (batch.cu): the internal order
// of the problems, each problem's block cap and workspace offsets in the
// device pool, and the static (problem, first row or column) tile lists that
// the step kernels walk.  Plain C++, no CUDA, so that its rules can be checked
// on a host without a GPU.
//
// Rules: problems are taken largest first (m n descending, ties in the caller's
// order), so their tiles are issued first and the hardware scheduler balances
// the tail; a problem stops after cap = ceil(min(m, n) / 2b) blocks (or
// max_blocks, if smaller; at least one), so its basis holds lmax = cap b
// columns; its buffers are laid out one after another, each starting on a
// 256-byte boundary; tiles cover its columns in 32s (norm partials), its rows in
// 128s (sketch, panel R^-1 products), the rows of A^T in 128s, and, with the
// tile shape of its class (BatchTiling), its columns and its basis columns in
// 64 tn (products X^T Y: A^T X, Q_j^T A; Q^T X) and its rows in 64 nn (row
// products A G, X - Q F).  Lists are in internal order; the three tunable ones
// are grouped by shape class first (class 0's problems, then class 1's, then
// class 2's, each in internal order), so that each class runs as one launch of
// the kernel instantiated for its tile shape.  The tiling changes only how the
// work is cut, not what any thread sums or in which order.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

namespace lra {

struct BatchTile {
  int prob;   // internal index of the problem
  int start;  // first row or column of the tile
};

// Buffers of one problem in the pool, in this order (bytes, before alignment):
// Q m lmax 4, B^T n lmax 4, X m b 4, W n b 4, (none), F lmax b 4, R^{-1} b b 4,
// Omega values b zmax 4, Omega rows b zmax 4, R diagonal b 8, column norms b 8, (none).
constexpr int BATCH_BUFFERS = 12;

// Tile shapes of the batched products by shape class (the autotuner's knobs):
// tn[c] columns per thread of the X^T Y products (64 threads, 64 tn[c] columns
// per tile) for problems of column class c, nn[c] rows per thread of the row
// products (64 nn[c] rows per tile) for row class c; each 1, 2 or 4.
struct BatchTiling {
  int tn[3];
  int nn[3];
};
constexpr int BATCH_CLASSES = 3;
inline BatchTiling batch_default_tiling() { return BatchTiling{{2, 2, 2}, {2, 2, 2}}; }
inline bool batch_tiling_valid(const BatchTiling& t) {
  for (int c = 0; c < BATCH_CLASSES; ++c)
    for (int v : {t.tn[c], t.nn[c]})
      if (v != 1 && v != 2 && v != 4) return false;
  return true;
}
// Column classes (by n): < 256, < 640, the rest; row classes (by m): < 384, < 1200, the rest.
inline int batch_tn_class(int64_t n) { return n < 256 ? 0 : n < 640 ? 1 : 2; }
inline int batch_nn_class(int64_t m) { return m < 384 ? 0 : m < 1200 ? 1 : 2; }

struct BatchProblemPlan {
  int cap, lmax;
  int64_t offs[BATCH_BUFFERS];
  int c32_first, c32_count;
  int ctn_first, ctn_count;  // this problem's tiles in the X^T Y list over its columns
  int g64_first, g64_count;  // its 64-column groups (the indicator's partial sums)
  int tn, nn;                // columns / rows per thread of its tiles
};

struct BatchPlan {
  std::vector<int> ord;    // internal index -> caller's index
  std::vector<int> order;  // caller's index -> internal index
  std::vector<BatchProblemPlan> prob;  // by internal index
  std::vector<BatchTile> c32, ctn, rm, rn, qtn, rnn;
  int ctn_off[4] = {}, qtn_off[4] = {}, rnn_off[4] = {};  // class c: [off[c], off[c + 1])
  int n_g64 = 0;  // 64-column groups of all problems
  int64_t pool_bytes = 0;
  int max_steps = 0;
};

inline int64_t batch_align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ms[i], ns[i]: the shape of problem i in the caller's order (validated by the
// caller: 1 <= b <= min(m, n)); b: block size; max_blocks: 0 or a cap on the
// blocks; zmax: the largest zeta the Omega buffers hold.
inline BatchPlan make_batch_plan(const std::vector<int64_t>& ms, const std::vector<int64_t>& ns,
                                 int b, int max_blocks, int zmax,
                                 const BatchTiling& tiling = batch_default_tiling()) {
  BatchPlan plan;
  const int count = (int)ms.size();
  plan.ord.resize(count);
  std::iota(plan.ord.begin(), plan.ord.end(), 0);
  std::stable_sort(plan.ord.begin(), plan.ord.end(),
                   [&](int x, int y) { return ms[x] * ns[x] > ms[y] * ns[y]; });
  plan.order.assign(count, 0);
  for (int k = 0; k < count; ++k) plan.order[plan.ord[k]] = k;
  plan.prob.resize(count);
  int64_t off = 0;
  for (int k = 0; k < count; ++k) {
    const int i = plan.ord[k];
    const int m = (int)ms[i], n = (int)ns[i];
    BatchProblemPlan& p = plan.prob[k];
    const int mn = std::min(m, n);
    int cap = (mn + 2 * b - 1) / (2 * b);
    if (max_blocks > 0) cap = std::min(cap, max_blocks);
    p.cap = std::max(cap, 1);
    p.lmax = p.cap * b;
    const int64_t sz[BATCH_BUFFERS] = {(int64_t)m * p.lmax * 4, (int64_t)n * p.lmax * 4,
                                       (int64_t)m * b * 4,      (int64_t)n * b * 4,
                                       0,                       (int64_t)p.lmax * b * 4,
                                       (int64_t)b * b * 4,      (int64_t)b * zmax * 4,
                                       (int64_t)b * zmax * 4,   (int64_t)b * 8,
                                       (int64_t)b * 8,          0};
    for (int q = 0; q < BATCH_BUFFERS; ++q) {
      p.offs[q] = off;
      off += batch_align_up(sz[q], 256);
    }
    p.c32_first = (int)plan.c32.size();
    for (int c0 = 0; c0 < n; c0 += 32) plan.c32.push_back(BatchTile{k, c0});
    p.c32_count = (int)plan.c32.size() - p.c32_first;
    p.g64_first = plan.n_g64;
    p.g64_count = (n + 63) / 64;
    plan.n_g64 += p.g64_count;
    p.tn = tiling.tn[batch_tn_class(n)];
    p.nn = tiling.nn[batch_nn_class(m)];
    for (int r0 = 0; r0 < m; r0 += 128) plan.rm.push_back(BatchTile{k, r0});
    for (int r0 = 0; r0 < n; r0 += 128) plan.rn.push_back(BatchTile{k, r0});
    plan.max_steps = std::max(plan.max_steps, p.cap);
  }
  // the tunable lists, class by class
  for (int c = 0; c < BATCH_CLASSES; ++c) {
    plan.ctn_off[c] = (int)plan.ctn.size();
    plan.qtn_off[c] = (int)plan.qtn.size();
    plan.rnn_off[c] = (int)plan.rnn.size();
    for (int k = 0; k < count; ++k) {
      const int i = plan.ord[k];
      const int m = (int)ms[i], n = (int)ns[i];
      BatchProblemPlan& p = plan.prob[k];
      if (batch_tn_class(n) == c) {
        p.ctn_first = (int)plan.ctn.size();
        for (int c0 = 0; c0 < n; c0 += 64 * p.tn) plan.ctn.push_back(BatchTile{k, c0});
        p.ctn_count = (int)plan.ctn.size() - p.ctn_first;
        for (int c0 = 0; c0 < p.lmax; c0 += 64 * p.tn) plan.qtn.push_back(BatchTile{k, c0});
      }
      if (batch_nn_class(m) == c)
        for (int r0 = 0; r0 < m; r0 += 64 * p.nn) plan.rnn.push_back(BatchTile{k, r0});
    }
  }
  plan.ctn_off[BATCH_CLASSES] = (int)plan.ctn.size();
  plan.qtn_off[BATCH_CLASSES] = (int)plan.qtn.size();
  plan.rnn_off[BATCH_CLASSES] = (int)plan.rnn.size();
  plan.pool_bytes = off;
  return plan;
}

}  // namespace lra
