// Randomised checks of the chunk schedules (csrc/chunk_schedule.h), host
// only:
//  1. leaf chunks: each pick equals the rule worked out here a second way
//     (sort the absent chunks by work, then decide), and it never names a
//     resident chunk;
//  2. leaf chunks, simulated calls: queries walk random chunk sequences
//     (mostly to a neighbouring chunk, as traversals move between nearby
//     leaves); a round scans the resident chunks holding queries and moves
//     each of their queries one visit on.  Every call ends, in no more
//     rounds than it has visits, with every visit made once, and the two
//     buffers never hold the same chunk;
//  3. point chunks: consecutive scans of a round use different buffers (the
//     next copy never waits for the scan before it), a chunk already
//     resident is never copied, and with every chunk holding queries every
//     round after the first copies exactly N - 2 chunks.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "chunk_schedule.h"

static int fails = 0;
static void check(bool ok, const char* what, long long at) {
  if (!ok && fails++ < 10) std::printf("FAIL %s at %lld\n", what, at);
}

// The leaf-chunk rule, restated: order the absent chunks holding queries by
// (most queries, lowest index); the first is the candidate.
static bkd::ChunkLoad rule(const std::vector<int64_t>& w, const int res[2]) {
  std::vector<int> absent;
  for (int c = 0; c < (int)w.size(); ++c)
    if (c != res[0] && c != res[1] && w[c] > 0) absent.push_back(c);
  bkd::ChunkLoad r;
  if (absent.empty()) return r;
  std::stable_sort(absent.begin(), absent.end(),
                   [&](int a, int b) { return w[a] > w[b]; });
  const int cand = absent[0];
  const int64_t w0 = res[0] >= 0 ? w[res[0]] : 0;
  const int64_t w1 = res[1] >= 0 ? w[res[1]] : 0;
  bool copy = false;
  int buf = -1;
  if (res[0] == -1) {
    copy = true;
    buf = 0;
  } else if (res[1] == -1) {
    copy = true;
    buf = 1;
  } else if (w0 + w1 == 0 || w[cand] > 2 * (w0 + w1)) {
    copy = true;
    buf = w1 < w0 ? 1 : 0;
  }
  if (copy) {
    r.buffer = buf;
    r.chunk = cand;
  }
  return r;
}

static void leaf_picks(std::mt19937_64& rng) {
  for (long long it = 0; it < 200000; ++it) {
    const int n = 1 + (int)(rng() % 12);
    std::vector<int64_t> w(n);
    for (auto& x : w) x = rng() % 3 == 0 ? 0 : (int64_t)(rng() % 50);
    int res[2] = {-1, -1};
    for (int b = 0; b < 2; ++b)
      if (rng() % 4) res[b] = (int)(rng() % n);
    if (res[0] == res[1]) res[1] = -1;  // a chunk is held at most once
    const bkd::ChunkLoad got =
        bkd::pick_leaf_chunk_load(n, res, [&](int c) { return w[c]; });
    const bkd::ChunkLoad want = rule(w, res);
    check(got.buffer == want.buffer && got.chunk == want.chunk,
          "leaf pick differs from the restated rule", it);
    if (got.buffer >= 0)
      check(got.chunk != res[0] && got.chunk != res[1] && w[got.chunk] > 0,
            "leaf pick names a resident or empty chunk", it);
  }
}

static void leaf_calls(std::mt19937_64& rng) {
  for (long long call = 0; call < 2000; ++call) {
    const int n = 1 + (int)(rng() % 10);
    const int nq = 1 + (int)(rng() % 300);
    std::vector<std::vector<int>> seq(nq);  // each query's chunks, in order
    int64_t visits = 0;
    for (auto& s : seq) {
      const int len = 1 + (int)(rng() % 40);
      int c = (int)(rng() % n);
      for (int j = 0; j < len; ++j) {
        s.push_back(c);
        const int r = (int)(rng() % 10);
        if (r < 6) continue;                       // same chunk
        if (r < 9) c = std::min(n - 1, std::max(0, c + (r == 6 ? -1 : 1)));
        else c = (int)(rng() % n);                 // anywhere
      }
      visits += len;
    }
    std::vector<size_t> pos(nq, 0);
    int res[2] = {-1, -1};
    int64_t rounds = 0, made = 0;
    for (;;) {
      std::vector<int64_t> w(n, 0);
      int64_t live = 0;
      for (int q = 0; q < nq; ++q)
        if (pos[q] < seq[q].size()) {
          ++w[seq[q][pos[q]]];
          ++live;
        }
      if (live == 0) break;
      ++rounds;
      if (rounds > visits) break;
      const bkd::ChunkLoad p =
          bkd::pick_leaf_chunk_load(n, res, [&](int c) { return w[c]; });
      if (p.buffer >= 0) res[p.buffer] = p.chunk;
      check(res[0] < 0 || res[0] != res[1], "one chunk in both buffers", call);
      int64_t moved = 0;
      for (int q = 0; q < nq; ++q)
        if (pos[q] < seq[q].size()) {
          const int c = seq[q][pos[q]];
          if (c == res[0] || c == res[1]) {
            ++pos[q];
            ++moved;
          }
        }
      check(moved > 0, "a round with buffered queries scans none", call);
      made += moved;
    }
    check(rounds <= visits, "more rounds than visits", call);
    check(made == visits, "visits made != visits", call);
  }
}

static void point_rounds(std::mt19937_64& rng) {
  for (long long call = 0; call < 2000; ++call) {
    const int n = 1 + (int)(rng() % 12);
    const bool all = rng() % 2;  // every chunk holds queries every round
    int res[2] = {-1, -1};
    for (int64_t round = 0; round < 30; ++round) {
      int prev_b = -1, copies = 0;
      std::vector<int> seen;
      for (int i = 0; i < n; ++i) {
        const int c = bkd::point_chunk_at(round, i, n);
        seen.push_back(c);
        if (!all && rng() % 3 == 0) continue;  // no queries there
        const int b = bkd::point_chunk_buffer(c, res, prev_b);
        check(b == 0 || b == 1, "point buffer out of range", call);
        check(prev_b < 0 || b != prev_b, "consecutive scans share a buffer",
              call);
        const bool held = res[0] == c || res[1] == c;
        if (held) check(res[b] == c, "a resident chunk copied again", call);
        if (res[b] != c) {
          res[b] = c;
          ++copies;
        }
        check(res[0] < 0 || res[0] != res[1], "one chunk in both buffers",
              call);
        prev_b = b;
      }
      std::sort(seen.begin(), seen.end());
      for (int i = 0; i < n; ++i)
        check(seen[i] == i, "a round does not visit every chunk once", call);
      if (all)
        check(copies == (round == 0 ? n : std::max(0, n - 2)),
              "copies per round with every chunk busy", call);
    }
  }
}

int main() {
  std::mt19937_64 rng(20151209);
  leaf_picks(rng);
  leaf_calls(rng);
  point_rounds(rng);
  if (fails) {
    std::printf("%d failures\n", fails);
    return 1;
  }
  std::printf("OK\n");
  return 0;
}
