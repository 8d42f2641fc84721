// Admission policy of the serving runtime (serve.cu): plain C++, no CUDA, so
// that its rules can be exercised on a host without a GPU.
//
// Requests wait in arrival order.  A free worker slot takes the oldest waiting
// request once its device-memory need fits under the budget next to what the
// running requests hold (first come, first served: a large request at the head
// is never overtaken, so it cannot starve).  A request whose need alone exceeds
// the budget is refused at submission.
#pragma once

#include <stdint.h>

#include <deque>
#include <utility>

namespace lra {

template <class Item>
class Admission {
 public:
  Admission(int64_t budget, int slots) : budget_(budget), slots_(slots) {}

  // false (and nothing queued) when the request can never fit.
  bool submit(Item item, int64_t bytes) {
    if (bytes < 0 || bytes > budget_) return false;
    queue_.push_back(Entry{std::move(item), bytes});
    return true;
  }

  // The next request to start, if a slot is free and the head of the queue fits;
  // its bytes are reserved until release().
  bool admit(Item* out, int64_t* bytes) {
    if (queue_.empty() || running_ >= slots_) return false;
    const Entry& head = queue_.front();
    if (held_ + head.bytes > budget_) return false;
    *out = std::move(queue_.front().item);
    *bytes = head.bytes;
    held_ += head.bytes;
    ++running_;
    queue_.pop_front();
    return true;
  }

  // A running request ends: its slot is free again and `returned` of its bytes
  // go back to the budget (the rest stay held, e.g. by a context kept for the
  // caller, until free_bytes()).
  void finish(int64_t returned) {
    held_ -= returned;
    --running_;
  }

  void free_bytes(int64_t bytes) { held_ -= bytes; }

  int64_t held() const { return held_; }
  int running() const { return running_; }
  size_t waiting() const { return queue_.size(); }
  int64_t budget() const { return budget_; }

 private:
  struct Entry {
    Item item;
    int64_t bytes;
  };
  int64_t budget_;
  int slots_;
  int64_t held_ = 0;
  int running_ = 0;
  std::deque<Entry> queue_;
};

}  // namespace lra
