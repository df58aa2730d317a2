// Randomised check of the server's slot allocator (csrc/slots.h) against a
// plain occupancy array: ranges never overlap, take() finds the lowest fit,
// give() merges, and with nothing taken the whole range is one block.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <utility>
#include <vector>

#include "slots.h"

static int fail(const char* what, int step) {
  std::printf("FAIL %s at step %d\n", what, step);
  return 1;
}

int main() {
  const int64_t n = 1000;
  std::mt19937_64 rng(12345);
  bkd::Slots s;
  s.reset(n);
  std::vector<char> used(n, 0);
  std::vector<std::pair<int64_t, int64_t>> live;
  for (int step = 0; step < 200000; ++step) {
    if (live.empty() || rng() % 2) {
      const int64_t len = 1 + (int64_t)(rng() % 120);
      // the lowest start with len free slots, from the occupancy array
      int64_t want = -1;
      for (int64_t a = 0, run = 0; a < n; ++a) {
        run = used[a] ? 0 : run + 1;
        if (run == len) { want = a - len + 1; break; }
      }
      const int64_t got = s.take(len);
      // first fit over maximal free blocks == lowest start of a long
      // enough run
      if (got != want) return fail("take", step);
      if (got >= 0) {
        for (int64_t a = got; a < got + len; ++a) used[a] = 1;
        live.push_back({got, len});
      }
    } else {
      const size_t i = rng() % live.size();
      s.give(live[i].first, live[i].second);
      for (int64_t a = live[i].first; a < live[i].first + live[i].second; ++a)
        used[a] = 0;
      live[i] = live.back();
      live.pop_back();
    }
    // the free map is exactly the free slots, blocks maximal
    int64_t prev_end = -2, total = 0;
    for (const auto& kv : s.free_) {
      if (kv.first <= prev_end) return fail("merge", step);
      for (int64_t a = kv.first; a < kv.first + kv.second; ++a)
        if (used[a]) return fail("overlap", step);
      prev_end = kv.first + kv.second;
      total += kv.second;
    }
    int64_t free_slots = 0;
    for (char u : used) free_slots += !u;
    if (total != free_slots) return fail("count", step);
  }
  for (auto& r : live) s.give(r.first, r.second);
  if (s.free_.size() != 1 || s.free_.begin()->first != 0 ||
      s.free_.begin()->second != n)
    return fail("coalesce", -1);
  std::printf("OK\n");
  return 0;
}
