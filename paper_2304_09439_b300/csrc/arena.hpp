// Host-side bookkeeping of the request server (plain C++, no CUDA): the
// allocator of the device arena that holds admitted requests, and the policy
// that packs the pairs of several requests into one launch.  Kept free of CUDA
// so that it compiles and is tested on a machine without a GPU.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace locc {

// First-fit allocator over the byte offsets [0, capacity) of one device
// buffer.  It hands out offsets only; the buffer itself belongs to the caller.
// Free blocks live in an ordered map (offset -> size) and are merged with
// their neighbours on release, so a fully released arena is one free block
// again.  Every block is a multiple of `align` bytes and starts on such a
// boundary.  Not thread-safe (the server holds its lock around every call).
class Arena {
 public:
  explicit Arena(size_t capacity = 0, size_t align = 256) { reset(capacity, align); }

  void reset(size_t capacity, size_t align = 256) {
    align_ = align ? align : 1;
    cap_ = capacity / align_ * align_;
    free_.clear();
    live_.clear();
    if (cap_) free_[0] = cap_;
    used_ = peak_ = 0;
  }

  size_t round(size_t bytes) const {
    const size_t b = bytes ? bytes : 1;
    return (b + align_ - 1) / align_ * align_;
  }

  // Whether a request of `bytes` could ever be served (alone in the arena).
  bool fits_empty(size_t bytes) const { return round(bytes) <= cap_; }

  // Lowest free offset with room for `bytes`; false (and *off untouched)
  // when no free block is large enough.
  bool alloc(size_t bytes, size_t* off) {
    const size_t need = round(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const size_t o = it->first, rest = it->second - need;
      free_.erase(it);
      if (rest) free_[o + need] = rest;
      live_[o] = need;
      used_ += need;
      peak_ = std::max(peak_, used_);
      *off = o;
      return true;
    }
    return false;
  }

  // Release a block returned by alloc; false for an offset that is not live.
  bool release(size_t off) {
    auto lv = live_.find(off);
    if (lv == live_.end()) return false;
    size_t o = off, n = lv->second;
    live_.erase(lv);
    used_ -= n;
    auto next = free_.lower_bound(o);
    if (next != free_.end() && o + n == next->first) {
      n += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == o) {
        o = prev->first;
        n += prev->second;
        free_.erase(prev);
      }
    }
    free_[o] = n;
    return true;
  }

  size_t capacity() const { return cap_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t n_live() const { return live_.size(); }
  size_t n_free_blocks() const { return free_.size(); }
  size_t largest_free() const {
    size_t m = 0;
    for (const auto& f : free_) m = std::max(m, f.second);
    return m;
  }
  // Free blocks in offset order, for invariant checks.
  const std::map<size_t, size_t>& free_blocks() const { return free_; }
  const std::map<size_t, size_t>& live_blocks() const { return live_; }

 private:
  size_t align_ = 256, cap_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_, live_;
};

// Pairs each active request contributes to the next launch of at most `cap`
// pairs.  remaining[i] = pairs of request i not yet dispatched, requests in
// admission order.  First every request gets up to an equal share
// (cap / n, at least 1 while room is left), so a small request admitted behind
// a large one finishes in the next launch instead of waiting for the large one
// to drain; then the room left is filled in admission order.  Writes take[i]
// and returns the total (<= cap, and == min(cap, sum of remaining)).
inline int64_t pack_launch(const int64_t* remaining, int n, int64_t cap, int64_t* take) {
  if (n <= 0 || cap <= 0) {
    for (int i = 0; i < n; ++i) take[i] = 0;
    return 0;
  }
  const int64_t share = std::max<int64_t>(1, cap / n);
  int64_t room = cap;
  for (int i = 0; i < n; ++i) {
    const int64_t t = std::min(std::max<int64_t>(remaining[i], 0), std::min(share, room));
    take[i] = t;
    room -= t;
  }
  for (int i = 0; i < n && room > 0; ++i) {
    const int64_t t = std::min(std::max<int64_t>(remaining[i], 0) - take[i], room);
    take[i] += t;
    room -= t;
  }
  return cap - room;
}

}  // namespace locc
