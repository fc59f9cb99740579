// fp_arena.h -- first-fit allocator of unit ranges, for the request server's
// device-memory budget.  Host-only C++ (no CUDA), so that it is also built
// and exercised on its own by the CPU tests.
//
// The arena hands out ranges [off, off + n) of [0, capacity).  Free ranges
// are kept ordered by offset and merged with their neighbours on release,
// so that a run of releases always restores one range per gap between live
// allocations.  First fit in offset order: the lowest free range that holds
// n units is split.  Not thread-safe: one owner calls it.
#pragma once

#include <cstdint>
#include <iterator>
#include <map>

namespace fp {

class Arena {
 public:
  explicit Arena(uint64_t capacity) : capacity_(capacity), free_units_(capacity) {
    if (capacity) free_[0] = capacity;
  }

  uint64_t capacity() const { return capacity_; }
  uint64_t free_units() const { return free_units_; }
  uint64_t used_units() const { return capacity_ - free_units_; }
  size_t fragments() const { return free_.size(); }

  uint64_t largest_free() const {
    uint64_t m = 0;
    for (const auto& kv : free_) m = kv.second > m ? kv.second : m;
    return m;
  }

  // Take n > 0 units; false (and nothing changed) when no free range holds n.
  bool alloc(uint64_t n, uint64_t* off) {
    if (n == 0) return false;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const uint64_t o = it->first, len = it->second;
      free_.erase(it);
      if (len > n) free_[o + n] = len - n;
      free_units_ -= n;
      *off = o;
      return true;
    }
    return false;
  }

  // Give back [off, off + n), a range that alloc returned (whole).
  void release(uint64_t off, uint64_t n) {
    if (n == 0) return;
    auto next = free_.lower_bound(off);
    uint64_t o = off, len = n;
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {  // merge with the range below
        o = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    if (next != free_.end() && next->first == off + n) {  // and with the one above
      len += next->second;
      free_.erase(next);
    }
    free_[o] = len;
    free_units_ += n;
  }

  // Visit the free ranges in offset order (for checks).
  template <class F>
  void for_each_free(F f) const {
    for (const auto& kv : free_) f(kv.first, kv.second);
  }

 private:
  uint64_t capacity_;
  uint64_t free_units_;
  std::map<uint64_t, uint64_t> free_;  // offset -> length, disjoint, never adjacent
};

}  // namespace fp
