// slots.h -- first-fit allocator of contiguous query-slot ranges (host
// only): the server admits a batch when a free range of its size exists and
// gives the range back when the batch completes.  Adjacent free ranges are
// merged, so with nothing in flight the whole range is one free block again.
#pragma once

#include <cstdint>
#include <iterator>
#include <map>

namespace bkd {

struct Slots {
  std::map<int64_t, int64_t> free_;  // start -> length; disjoint, and no
                                     // two adjacent (neighbours merge)
  // all of [0, n) free
  void reset(int64_t n) {
    free_.clear();
    if (n > 0) free_[0] = n;
  }
  // first (lowest) start of a free range of `len` slots, now taken; -1 if
  // none is large enough
  int64_t take(int64_t len) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < len) continue;
      const int64_t s = it->first, rest = it->second - len;
      free_.erase(it);
      if (rest > 0) free_[s + len] = rest;
      return s;
    }
    return -1;
  }
  // returns [s, s + len), taken before, merging it with free neighbours
  void give(int64_t s, int64_t len) {
    auto it = free_.emplace(s, len).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace bkd
