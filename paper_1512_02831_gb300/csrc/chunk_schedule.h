// chunk_schedule.h -- which chunk of a chunked leaf structure goes into
// which of the two device chunk buffers (host only; the Brute / Copy / Wait
// cycle of Sec. 3.2 over chunks held in pinned host memory, Sec. 3).
//
// Leaf chunks (whole leaves per chunk): the residency schedule.  Before a
// round's ProcessAllBuffers, work(c) is the number of queries buffered in
// the leaves of chunk c and resident[b] the chunk held by device buffer b
// (-1: empty).  The absent chunk with the most buffered queries (the lowest
// index among equals) is copied in when a buffer is empty (buffer 0 first),
// when the resident chunks hold no buffered query, or when it holds more
// than twice their queries together; it then replaces the resident chunk
// with fewer buffered queries (buffer 0 among equals).  Otherwise nothing
// is copied.  The round scans the resident chunks that hold queries; those
// buffered in absent chunks wait for a later round.  Every round with
// buffered queries scans at least one of them (a resident chunk that holds
// some, or the chunk just copied in, which holds the most), so the rounds
// of a call are bounded by its leaf visits whatever the schedule does.
//
// Point chunks (the paper's chunk bounds, a leaf may straddle two chunks):
// every chunk that holds buffered queries is scanned each round, in
// ascending order in even rounds and descending order in odd ones, so the
// two chunks scanned last stay resident for the next round.  A chunk that
// is not resident goes into the buffer the previous scan of the round did
// not use (the first one: buffer 0 if it is empty, else buffer 1), so the
// copy of the next chunk overlaps the scan of the current one.
#pragma once

#include <cstdint>

namespace bkd {

struct ChunkLoad {
  int buffer = -1;  // the device buffer that receives a chunk; -1: no copy
  int chunk = -1;   // the chunk copied into it
};

// Leaf chunks: the copy (if any) before this round's scans.  `work(c)`
// returns the buffered queries of chunk c (c in [0, n_chunks)).
template <class Work>
inline ChunkLoad pick_leaf_chunk_load(int n_chunks, const int resident[2],
                                      Work work) {
  auto held = [&](int c) { return c < 0 ? int64_t(0) : int64_t(work(c)); };
  int best = -1;
  for (int c = 0; c < n_chunks; ++c)
    if (c != resident[0] && c != resident[1] && held(c) > 0 &&
        (best < 0 || held(c) > held(best)))
      best = c;
  ChunkLoad r;
  if (best < 0) return r;
  const int64_t wres = held(resident[0]) + held(resident[1]);
  if (resident[0] < 0)
    r.buffer = 0;
  else if (resident[1] < 0)
    r.buffer = 1;
  else if (wres == 0 || held(best) > 2 * wres)
    r.buffer = held(resident[0]) <= held(resident[1]) ? 0 : 1;
  if (r.buffer >= 0) r.chunk = best;
  return r;
}

// Point chunks: the chunk scanned i-th (i in [0, n_chunks)) in `round`.
inline int point_chunk_at(int64_t round, int i, int n_chunks) {
  return round % 2 == 0 ? i : n_chunks - 1 - i;
}

// Point chunks: the buffer chunk c is scanned from; `prev_b` is the buffer
// of the round's previous scan (-1: c is the round's first).  The caller
// copies c into it unless resident[buffer] == c already.
inline int point_chunk_buffer(int c, const int resident[2], int prev_b) {
  if (resident[0] == c) return 0;
  if (resident[1] == c) return 1;
  if (prev_b < 0) return resident[0] == -1 ? 0 : 1;
  return 1 - prev_b;
}

}  // namespace bkd
