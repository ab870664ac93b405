// Host-side policy of the serving form, free of CUDA so that it builds and is
// tested with a plain C++ compiler:
//   * Arena: first-fit allocator over one device region (the HBM budget),
//     256-byte granules, neighbouring free ranges merged on release;
//   * AdmissionQueue: FIFO of submitted jobs; the head is admitted while a
//     slot is free and its footprint fits the arena, and nothing behind the
//     head is admitted ahead of it (arrival order is service order).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <deque>
#include <iterator>
#include <map>

namespace ntt {
namespace serve {

class Arena {
 public:
  static constexpr size_t kAlign = 256;
  explicit Arena(size_t bytes = 0) { reset(bytes); }

  void reset(size_t bytes) {
    free_.clear();
    used_.clear();
    capacity_ = bytes / kAlign * kAlign;
    in_use_ = peak_ = 0;
    if (capacity_) free_[0] = capacity_;
  }

  // Offset of a block of at least `bytes`, or -1 when no free range holds it.
  int64_t alloc(size_t bytes) {
    const size_t need = (bytes + kAlign - 1) / kAlign * kAlign;
    if (need == 0) return -1;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > need) free_[off + need] = len - need;
      used_[off] = need;
      in_use_ += need;
      if (in_use_ > peak_) peak_ = in_use_;
      return (int64_t)off;
    }
    return -1;
  }

  // Release a block returned by alloc; false when `off` is not a live block.
  bool release(int64_t off) {
    auto u = used_.find((size_t)off);
    if (off < 0 || u == used_.end()) return false;
    size_t start = u->first, len = u->second;
    used_.erase(u);
    in_use_ -= len;
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + len) {
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        prev->second += len;
        return true;
      }
    }
    free_[start] = len;
    return true;
  }

  size_t capacity() const { return capacity_; }
  size_t in_use() const { return in_use_; }
  size_t peak() const { return peak_; }
  size_t free_ranges() const { return free_.size(); }
  size_t largest_free() const {
    size_t b = 0;
    for (const auto& f : free_) b = f.second > b ? f.second : b;
    return b;
  }

 private:
  std::map<size_t, size_t> free_;   // offset -> length
  std::map<size_t, size_t> used_;
  size_t capacity_ = 0, in_use_ = 0, peak_ = 0;
};

struct Pending {
  int64_t id;
  size_t footprint;
};

class AdmissionQueue {
 public:
  void push(int64_t id, size_t footprint) { q_.push_back({id, footprint}); }
  size_t size() const { return q_.size(); }
  bool empty() const { return q_.empty(); }

  // Admit from the head while a slot is free and the arena takes the head's
  // footprint; `admit(id, offset)` receives each admitted job.  Returns the
  // number admitted.  A head larger than the whole arena is returned through
  // `reject` (it can never run) and the next job becomes the head.
  template <class Admit, class Reject>
  int admit(Arena& arena, int free_slots, Admit admit_fn, Reject reject_fn) {
    int n = 0;
    while (!q_.empty() && free_slots > 0) {
      const Pending h = q_.front();
      if (h.footprint > arena.capacity()) {
        q_.pop_front();
        reject_fn(h.id);
        continue;
      }
      const int64_t off = arena.alloc(h.footprint);
      if (off < 0) break;   // wait for releases; keep arrival order
      q_.pop_front();
      admit_fn(h.id, off);
      --free_slots;
      ++n;
    }
    return n;
  }

 private:
  std::deque<Pending> q_;
};

}  // namespace serve
}  // namespace ntt
