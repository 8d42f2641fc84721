// Host-side checks of the batched form's plan (batch_plan.h): order, block
// caps, pool layout and tile lists.  Prints one word pair per check; exits
// non-zero on the first failure.
#include <stdio.h>
#include <stdlib.h>

#include <random>
#include <vector>

#include "batch_plan.h"

#define CHECK(c)                                                      \
  do {                                                                \
    if (!(c)) {                                                       \
      fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__);  \
      exit(1);                                                        \
    }                                                                 \
  } while (0)

using lra::BatchPlan;
using lra::BatchTile;

// Buffer sizes as the plan's header states them.
static void sizes(int64_t m, int64_t n, int64_t lmax, int64_t b, int64_t zmax, int64_t* sz) {
  const int64_t s[lra::BATCH_BUFFERS] = {m * lmax * 4, n * lmax * 4, m * b * 4, n * b * 4, 0, lmax * b * 4,
                                         b * b * 4,    b * zmax * 4, b * zmax * 4, b * 8,  b * 8, 0};
  for (int q = 0; q < lra::BATCH_BUFFERS; ++q) sz[q] = s[q];
}

// Tiles of problem k in list L, in order: starts 0, step, 2 step, ... below extent.
static void covers(const std::vector<BatchTile>& L, int k, int extent, int step) {
  int next = 0;
  for (const BatchTile& t : L) {
    if (t.prob != k) continue;
    CHECK(t.start == next);
    next += step;
  }
  CHECK(next >= extent && next - step < extent);
}

static void check_plan(const std::vector<int64_t>& ms, const std::vector<int64_t>& ns, int b, int max_blocks,
                       int zmax, const lra::BatchTiling& tl = lra::batch_default_tiling()) {
  const int count = (int)ms.size();
  const BatchPlan p = lra::make_batch_plan(ms, ns, b, max_blocks, zmax, tl);
  // order: a permutation, largest first, ties in the caller's order; order is its inverse
  CHECK((int)p.ord.size() == count && (int)p.order.size() == count);
  std::vector<int> seen(count, 0);
  for (int k = 0; k < count; ++k) {
    CHECK(p.ord[k] >= 0 && p.ord[k] < count && !seen[p.ord[k]]);
    seen[p.ord[k]] = 1;
    CHECK(p.order[p.ord[k]] == k);
    if (k > 0) {
      const int64_t a = ms[p.ord[k - 1]] * ns[p.ord[k - 1]], c = ms[p.ord[k]] * ns[p.ord[k]];
      CHECK(a > c || (a == c && p.ord[k - 1] < p.ord[k]));
    }
  }
  // caps, pool layout, tile lists
  int64_t end = 0;
  int max_cap = 0;
  for (int k = 0; k < count; ++k) {
    const int64_t m = ms[p.ord[k]], n = ns[p.ord[k]];
    const lra::BatchProblemPlan& q = p.prob[k];
    int cap = (int)((std::min(m, n) + 2 * b - 1) / (2 * b));
    if (max_blocks > 0 && max_blocks < cap) cap = max_blocks;
    if (cap < 1) cap = 1;
    CHECK(q.cap == cap && q.lmax == cap * b);
    max_cap = std::max(max_cap, cap);
    int64_t sz[lra::BATCH_BUFFERS];
    sizes(m, n, q.lmax, b, zmax, sz);
    for (int j = 0; j < lra::BATCH_BUFFERS; ++j) {
      CHECK(q.offs[j] % 256 == 0);
      CHECK(q.offs[j] >= end);  // after every earlier buffer: no overlap
      end = q.offs[j] + sz[j];
    }
    // the tile shape of the problem's class
    CHECK(q.tn == tl.tn[lra::batch_tn_class(n)] && q.nn == tl.nn[lra::batch_nn_class(m)]);
    const int wtn = 64 * q.tn, wnn = 64 * q.nn;
    covers(p.c32, k, (int)n, 32);
    covers(p.ctn, k, (int)n, wtn);
    covers(p.rm, k, (int)m, 128);
    covers(p.rn, k, (int)n, 128);
    covers(p.qtn, k, q.lmax, wtn);
    covers(p.rnn, k, (int)m, wnn);
    CHECK(q.c32_count == (int)((n + 31) / 32) && q.ctn_count == (int)((n + wtn - 1) / wtn));
    for (int t = 0; t < q.c32_count; ++t) CHECK(p.c32[q.c32_first + t].prob == k);
    for (int t = 0; t < q.ctn_count; ++t) CHECK(p.ctn[q.ctn_first + t].prob == k);
    CHECK(q.g64_count == (int)((n + 63) / 64) && q.g64_first == (k ? p.prob[k - 1].g64_first + p.prob[k - 1].g64_count : 0));
  }
  CHECK(p.pool_bytes >= end && p.pool_bytes % 256 == 0 && p.max_steps == max_cap);
  // the tiling changes neither the order nor the pool
  const BatchPlan d = lra::make_batch_plan(ms, ns, b, max_blocks, zmax);
  CHECK(d.ord == p.ord && d.pool_bytes == p.pool_bytes && d.n_g64 == p.n_g64);
  for (int k = 0; k < count; ++k) CHECK(d.prob[k].g64_first == p.prob[k].g64_first);
  CHECK(p.n_g64 <= (int)p.c32.size());
  // every list walks the problems in internal order; the tunable ones within each
  // shape class, whose sections hold exactly that class's problems
  for (const std::vector<BatchTile>* L : {&p.c32, &p.rm, &p.rn})
    for (size_t i = 1; i < L->size(); ++i) CHECK((*L)[i - 1].prob <= (*L)[i].prob);
  struct Sec {
    const std::vector<BatchTile>* L;
    const int* off;
    bool by_n;
  };
  for (const Sec& sec : {Sec{&p.ctn, p.ctn_off, true}, Sec{&p.qtn, p.qtn_off, true}, Sec{&p.rnn, p.rnn_off, false}}) {
    CHECK(sec.off[0] == 0 && sec.off[lra::BATCH_CLASSES] == (int)sec.L->size());
    for (int c = 0; c < lra::BATCH_CLASSES; ++c) {
      CHECK(sec.off[c] <= sec.off[c + 1]);
      for (int i = sec.off[c]; i < sec.off[c + 1]; ++i) {
        const int k = (*sec.L)[i].prob;
        const int64_t ext = sec.by_n ? ns[p.ord[k]] : ms[p.ord[k]];
        CHECK((sec.by_n ? lra::batch_tn_class(ext) : lra::batch_nn_class(ext)) == c);
        if (i > sec.off[c]) CHECK((*sec.L)[i - 1].prob <= k);
      }
    }
  }
}

int main() {
  // 1. fixed cases: edge shapes, ties, a cap from max_blocks
  check_plan({64, 2048, 100, 1000, 2048, 65, 513}, {32, 1024, 700, 32, 33, 1024, 257}, 16, 0, 16);
  check_plan({300, 300, 300}, {200, 200, 200}, 8, 0, 16);
  check_plan({1500, 64}, {900, 32}, 32, 2, 16);
  {
    const BatchPlan p = lra::make_batch_plan({100, 1000}, {50, 500}, 16, 0, 16);
    CHECK(p.ord[0] == 1 && p.ord[1] == 0);  // the larger problem first
    CHECK(p.prob[0].cap == 16 && p.prob[1].cap == 2);  // ceil(500 / 32), ceil(50 / 32)
  }
  printf("fixed ok\n");
  // 2. random batches
  std::mt19937_64 g(11);
  for (int trial = 0; trial < 500; ++trial) {
    const int count = 1 + (int)(g() % 80);
    const int b = (int[]){8, 16, 32}[g() % 3];
    const int max_blocks = (g() % 3 == 0) ? (int)(g() % 6) : 0;
    std::vector<int64_t> ms(count), ns(count);
    for (int i = 0; i < count; ++i) {
      ms[i] = b + (int64_t)(g() % 2100);
      ns[i] = b + (int64_t)(g() % 1100);
      if (i > 0 && g() % 6 == 0) {
        ms[i] = ms[i - 1];
        ns[i] = ns[i - 1];
      }
    }
    check_plan(ms, ns, b, max_blocks, 16);
    lra::BatchTiling tl;
    for (int c = 0; c < lra::BATCH_CLASSES; ++c) {
      tl.tn[c] = (int[]){1, 2, 4}[g() % 3];
      tl.nn[c] = (int[]){1, 2, 4}[g() % 3];
    }
    CHECK(lra::batch_tiling_valid(tl));
    check_plan(ms, ns, b, max_blocks, 16, tl);
  }
  CHECK(!lra::batch_tiling_valid(lra::BatchTiling{{2, 3, 2}, {2, 2, 2}}));
  printf("random ok\n");
  return 0;
}
