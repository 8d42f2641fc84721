// Host-side checks of the serving runtime's admission policy (serve_policy.h).
// Prints one line per check; exits non-zero on the first failure.
#include <stdio.h>
#include <stdlib.h>

#include <random>
#include <vector>

#include "serve_policy.h"

#define CHECK(c)                                                  \
  do {                                                            \
    if (!(c)) {                                                   \
      fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
      exit(1);                                                    \
    }                                                             \
  } while (0)

int main() {
  // 1. oversize requests are refused; FIFO admission; head of line is not overtaken
  {
    lra::Admission<int> a(100, 4);
    CHECK(!a.submit(0, 101));
    CHECK(a.submit(1, 60));
    CHECK(a.submit(2, 60));   // does not fit beside 1
    CHECK(a.submit(3, 10));   // would fit, but waits behind 2
    int it;
    int64_t b;
    CHECK(a.admit(&it, &b) && it == 1 && b == 60);
    CHECK(!a.admit(&it, &b));           // 2 is at the head and does not fit
    CHECK(a.waiting() == 2 && a.held() == 60);
    a.finish(60);
    CHECK(a.admit(&it, &b) && it == 2);
    CHECK(a.admit(&it, &b) && it == 3);
    CHECK(a.held() == 70 && a.running() == 2);
    printf("fifo ok\n");
  }
  // 2. the slot limit
  {
    lra::Admission<int> a(1000, 2);
    for (int i = 0; i < 5; ++i) CHECK(a.submit(i, 1));
    int it;
    int64_t b;
    CHECK(a.admit(&it, &b) && a.admit(&it, &b) && !a.admit(&it, &b));
    a.finish(1);
    CHECK(a.admit(&it, &b) && it == 2);
    printf("slots ok\n");
  }
  // 3. a kept context frees its slot but keeps its bytes until free_bytes
  {
    lra::Admission<int> a(100, 1);
    CHECK(a.submit(1, 70) && a.submit(2, 50));
    int it;
    int64_t b;
    CHECK(a.admit(&it, &b) && it == 1);
    a.finish(0);
    CHECK(a.running() == 0 && a.held() == 70);
    CHECK(!a.admit(&it, &b));  // 50 does not fit beside the kept 70
    a.free_bytes(70);
    CHECK(a.admit(&it, &b) && it == 2);
    printf("kept ok\n");
  }
  // 4. random trace: limits always hold, everything is admitted in order, and
  //    the queue drains
  {
    std::mt19937_64 rng(7);
    const int64_t budget = 1000;
    const int slots = 3;
    lra::Admission<int> a(budget, slots);
    struct Run {
      int id;
      int64_t bytes;
    };
    std::vector<Run> running;
    int next_id = 0, expect = 0, finished = 0;
    const int total = 5000;
    while (finished < total) {
      if (next_id < total && rng() % 2) {
        const int64_t bytes = 1 + (int64_t)(rng() % budget);
        CHECK(a.submit(next_id++, bytes));
      }
      int it;
      int64_t b;
      while (a.admit(&it, &b)) {
        CHECK(it == expect++);
        running.push_back({it, b});
      }
      CHECK(a.held() <= budget && a.running() <= slots && a.running() == (int)running.size());
      if (!running.empty() && (rng() % 2 || next_id == total)) {
        const size_t k = rng() % running.size();
        a.finish(running[k].bytes);
        running.erase(running.begin() + k);
        ++finished;
      }
    }
    CHECK(a.waiting() == 0 && a.held() == 0 && expect == total);
    printf("random ok\n");
  }
  return 0;
}
