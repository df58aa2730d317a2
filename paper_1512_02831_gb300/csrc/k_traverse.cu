// k_traverse.cu -- query initialisation and FindLeafBatch (Algorithm 1).
//
// FindLeafBatch continues each query's implicit tree traversal (Sec. 2.4)
// to the next leaf it has to visit, or reports -1 once the traversal has
// reached the root twice.  The traversal is the classical k-d tree search of
// Sec. 2.3: walk down to the cell containing q; on the way back up, visit the
// far child of a node iff it could still hold a better candidate, otherwise
// prune.
//
// The traversal step itself (stackless, exact bounding-box pruning) is
// next_leaf() in traverse.cuh, shared with the tail and fallback kernels.
#include <algorithm>

#include "bkd_internal.h"
#include "traverse.cuh"

namespace bkd {
namespace {

__global__ void init_kernel(const float* __restrict__ Q, int64_t m, int d,
                            int Dp, float* __restrict__ qpad,
                            float* __restrict__ lst_d,
                            uint32_t* __restrict__ lst_i, int K,
                            uint64_t* __restrict__ state,
                            uint32_t* __restrict__ act, uint32_t act_base,
                            Counters* ctr) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  bool bad = false;
  for (int i = 0; i < Dp; ++i) {
    float x = i < d ? Q[q * d + i] : 0.f;
    // finite and |x| < 2^60 keeps every squared difference finite
    bad |= !(fabsf(x) < 1.152921504606846976e18f);
    qpad[q * Dp + i] = x;
  }
  for (int j = 0; j < K; ++j) {
    lst_d[q * K + j] = __int_as_float(0x7f800000);  // +inf
    lst_i[q * K + j] = kNoSlot;
  }
  state[q] = trav_state(kStart, 0u);
  act[q] = act_base + (uint32_t)q;
  if (bad) atomicOr(&ctr->err, kErrNonFinite);
}

// One warp per CTA: traversal lengths differ from warp to warp, and a warp
// that finishes frees its slot at once instead of waiting for the other
// warps of its CTA (measured on the 2^24-point mixture: 21.9 ms per call
// against 25.3 ms with 128-thread and 64-thread CTAs).
constexpr int kFindThreads = 32;

// One thread per active query.  The active list is ordered by leaf (the
// previous round's scatter), so the lanes of a warp start from the same
// leaf and mostly test the same boxes at the same time.  (Persistent lanes
// that take a new query as soon as theirs is done were measured slower:
// they lose that locality.)  For the same reason most lanes of a warp count
// their query into the same few leaves: the count is warp-aggregated, one
// atomic per distinct leaf, each lane's rank from its place among the
// lanes of that leaf (the order inside a buffer is irrelevant).
template <int D>
__global__ void __launch_bounds__(kFindThreads)
    find_leaf_kernel(DevTree t, const float* __restrict__ qpad,
                     const uint32_t* __restrict__ act, int n_act,
                     const int32_t* __restrict__ n_act_dev,
                     uint64_t* __restrict__ state,
                     const float* __restrict__ lst_d, int K,
                     int2* __restrict__ placed,
                     int32_t* __restrict__ cnt) {
  static_assert(kFindThreads == 32, "one warp per CTA: the count below");
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x;
  const int first_leaf = (1 << t.h) - 1;
  int leaf_out = -1;  // the leaf this query is counted into (-1: none)
  if (pos < (n_act_dev ? *n_act_dev : n_act)) {
    const uint32_t q = act[pos];
    const float* qp = qpad + (size_t)q * D;
    const uint64_t st = state[q];
    const int node = state_node(st);
    uint32_t mask = state_mask(st);
    bool waits = false;  // the pending leaf is still to scan: stay there
    if (node >= 0) {
      // a deferred buffer (servers), or a chunk not scanned last round
      // (chunked mode)
      if (t.q_wait && t.q_wait[q]) waits = true;
      if (t.chunk_done &&
          !t.chunk_done[(int)(((int64_t)(node - first_leaf) * t.n_chunks) >>
                              t.h)])
        waits = true;
    }
    if (waits) {
      leaf_out = node - first_leaf;
    } else {
      const float bound = node == kStart ? __int_as_float(0x7f800000)
                                         : lst_d[(size_t)q * K + (K - 1)];
      F32Bound<D> bx;
      bx.load(qp);
      const int next = next_leaf(t, bx, qp, node, mask, bound);
      state[q] = trav_state(next, mask);
      if (next == kDone)
        placed[pos] = make_int2(-1, 0);
      else
        leaf_out = next - first_leaf;
    }
  }
  // every lane of the warp arrives here
  const unsigned peers = __match_any_sync(0xffffffffu, leaf_out);
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (leaf_out >= 0 && lane == leader)
    base = atomicAdd(cnt + leaf_out, __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (leaf_out >= 0)
    placed[pos] =
        make_int2(leaf_out, base + __popc(peers & ((1u << lane) - 1u)));
}

// ------------------------------------------------------------- bucketing
// Buffer insertion of Algorithm 1 as a counting sort by leaf id: the
// histogram is counted where the next leaf is found (FindLeafBatch, which
// also keeps each query's rank among the queries of its leaf); here follow
// the exclusive scan (also of per-leaf work items of `tile` queries) and the
// scatter to offset + rank.
// The order of queries inside a leaf's buffer is irrelevant to the results.

// Two-pass scan over the leaves, 2,048 leaves (8 per thread) per block:
// scan_parts_kernel sums each tile, scan_write_kernel adds the sums of the
// tiles before it and writes the offsets, the work items and the totals.
constexpr int kScanBlock = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanBlock * kScanPer;

struct ScanPart {
  int32_t q, t;                // queries and work items of the tile
  unsigned long long p;        // (query, point) pairs of the tile
};

__device__ __forceinline__ void tile_sums(const int32_t* __restrict__ cnt,
                                          int L, int tile,
                                          const int32_t* __restrict__ leaf_cnt,
                                          int lo, int32_t& q, int32_t& t,
                                          unsigned long long& p) {
  q = 0;
  t = 0;
  p = 0;
  const int hi = min(L, lo + kScanPer);
  for (int l = lo; l < hi; ++l) {
    const int c = cnt[l];
    q += c;
    t += (c + tile - 1) / tile;
    p += (unsigned long long)c * (unsigned long long)leaf_cnt[l];
  }
}

__global__ void __launch_bounds__(kScanBlock)
    scan_parts_kernel(const int32_t* __restrict__ cnt, int L, int tile,
                      const int32_t* __restrict__ leaf_cnt,
                      ScanPart* __restrict__ parts) {
  __shared__ int32_t sq[kScanBlock / 32], st[kScanBlock / 32];
  __shared__ unsigned long long sp[kScanBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t q, t;
  unsigned long long p;
  tile_sums(cnt, L, tile, leaf_cnt,
            blockIdx.x * kScanTile + threadIdx.x * kScanPer, q, t, p);
  for (int o = 16; o > 0; o >>= 1) {
    q += __shfl_down_sync(0xffffffffu, q, o);
    t += __shfl_down_sync(0xffffffffu, t, o);
    p += __shfl_down_sync(0xffffffffu, p, o);
  }
  if (lane == 0) {
    sq[warp] = q;
    st[warp] = t;
    sp[warp] = p;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ScanPart r{0, 0, 0};
    for (int w = 0; w < kScanBlock / 32; ++w) {
      r.q += sq[w];
      r.t += st[w];
      r.p += sp[w];
    }
    parts[blockIdx.x] = r;
  }
}

__global__ void __launch_bounds__(kScanBlock)
    scan_write_kernel(const int32_t* __restrict__ cnt, int L, int tile,
                      const int32_t* __restrict__ leaf_cnt,
                      const ScanPart* __restrict__ parts,
                      int32_t* __restrict__ off, int32_t* __restrict__ toff,
                      Item* __restrict__ items, Counters* ctr,
                      int32_t* __restrict__ n_next_dev) {
  __shared__ int32_t wq[kScanBlock / 32], wt[kScanBlock / 32];
  __shared__ int32_t bq0, bt0;
  __shared__ unsigned long long ptot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool last = blockIdx.x == gridDim.x - 1;
  // prefix of the tiles before this one (and, in the last block, the pairs
  // of all tiles)
  if (warp == 0) {
    int32_t q = 0, t = 0;
    unsigned long long p = 0;
    const int np = last ? gridDim.x : blockIdx.x;
    for (int j = lane; j < np; j += 32) {
      if (j < (int)blockIdx.x) {
        q += parts[j].q;
        t += parts[j].t;
      }
      p += parts[j].p;
    }
    for (int o = 16; o > 0; o >>= 1) {
      q += __shfl_down_sync(0xffffffffu, q, o);
      t += __shfl_down_sync(0xffffffffu, t, o);
      p += __shfl_down_sync(0xffffffffu, p, o);
    }
    if (lane == 0) {
      bq0 = q;
      bt0 = t;
      ptot = p;
    }
  }
  const int lo = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  int32_t q, t;
  unsigned long long p;
  tile_sums(cnt, L, tile, leaf_cnt, lo, q, t, p);
  int32_t iq = q, it = t;  // inclusive warp scans
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t a = __shfl_up_sync(0xffffffffu, iq, o);
    const int32_t b = __shfl_up_sync(0xffffffffu, it, o);
    if (lane >= o) {
      iq += a;
      it += b;
    }
  }
  if (lane == 31) {
    wq[warp] = iq;
    wt[warp] = it;
  }
  __syncthreads();
  int32_t xq = bq0, xt = bt0;  // exclusive prefix of this thread
  for (int w = 0; w < warp; ++w) {
    xq += wq[w];
    xt += wt[w];
  }
  xq += iq - q;
  xt += it - t;
  const int hi = min(L, lo + kScanPer);
  for (int l = lo; l < hi; ++l) {
    const int c = cnt[l];
    const int nt = (c + tile - 1) / tile;
    off[l] = xq;
    toff[l] = xt;
    for (int j = 0; j < nt; ++j) {
      Item w;
      w.leaf = l;
      w.start = xq + j * tile;
      w.count = min(tile, c - j * tile);
      w.pad = 0;
      items[xt + j] = w;
    }
    xq += c;
    xt += nt;
  }
  if (last && threadIdx.x == kScanBlock - 1) {
    off[L] = xq;
    toff[L] = xt;
    ctr->n_next = xq;
    ctr->n_items = xt;
    ctr->pairs = ptot;
    ctr->rounds_pairs += ptot;
    ctr->rounds_visits += (unsigned long long)xq;
    ctr->rounds_items += (unsigned long long)xt;
    if (xq > 0) ctr->rounds_run += 1;
    if (n_next_dev) *n_next_dev = xq;
  }
}

__global__ void scatter_kernel(const int2* __restrict__ placed,
                               const uint32_t* __restrict__ act, int n,
                               const int32_t* __restrict__ n_dev,
                               const int32_t* __restrict__ off,
                               uint32_t* __restrict__ next) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= (n_dev ? *n_dev : n)) return;
  const int2 p = placed[pos];
  if (p.x < 0) return;
  next[off[p.x] + p.y] = act[pos];
}

__global__ void chunk_items_kernel(const int32_t* __restrict__ toff,
                                   const int32_t* __restrict__ off,
                                   const int32_t* __restrict__ leaf,
                                   int count, int32_t* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < count) {
    out[c] = toff[leaf[c]];
    out[count + c] = off[leaf[c]];
  }
}

__global__ void fill_kernel(int32_t* __restrict__ v, int64_t n,
                            int32_t value) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = value;
}

// One less in its batch's count for every query that finished this round.
__global__ void retire_kernel(const int2* __restrict__ placed,
                              const uint32_t* __restrict__ act, int n,
                              const int32_t* __restrict__ slot_batch,
                              int32_t* __restrict__ batch_left) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= n || placed[pos].x >= 0) return;
  atomicSub(batch_left + slot_batch[act[pos]], 1);
}

// One less in its batch's count for every query of the list (all of them
// finished, e.g. by the tail kernel).
__global__ void retire_list_kernel(const uint32_t* __restrict__ act, int n,
                                   const int32_t* __restrict__ slot_batch,
                                   int32_t* __restrict__ batch_left) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= n) return;
  atomicSub(batch_left + slot_batch[act[pos]], 1);
}

inline int blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_fill(int32_t* v, int64_t n, int32_t value, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  fill_kernel<<<blocks(n, 256), 256, 0, s>>>(v, n, value);
  return cudaGetLastError();
}

cudaError_t launch_retire(const int2* placed, const uint32_t* act, int n_act,
                          const int32_t* slot_batch, int32_t* batch_left,
                          cudaStream_t s) {
  if (n_act <= 0) return cudaSuccess;
  retire_kernel<<<blocks(n_act, 256), 256, 0, s>>>(placed, act, n_act,
                                                   slot_batch, batch_left);
  return cudaGetLastError();
}

cudaError_t launch_retire_list(const uint32_t* act, int n,
                               const int32_t* slot_batch, int32_t* batch_left,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  retire_list_kernel<<<blocks(n, 256), 256, 0, s>>>(act, n, slot_batch,
                                                    batch_left);
  return cudaGetLastError();
}

cudaError_t launch_init(const float* Q, int64_t m, int d, int Dp, float* qpad,
                        float* lst_d, uint32_t* lst_i, int K, uint64_t* state,
                        uint32_t* act, uint32_t act_base, Counters* ctr,
                        cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  init_kernel<<<blocks(m, 256), 256, 0, s>>>(Q, m, d, Dp, qpad, lst_d, lst_i,
                                             K, state, act, act_base, ctr);
  return cudaGetLastError();
}

cudaError_t launch_find_leaf(const DevTree& t, const float* qpad,
                             const uint32_t* act, int n_act, uint64_t* state,
                             const float* lst_d, int K, int2* placed,
                             int32_t* cnt, cudaStream_t s,
                             const int32_t* n_act_dev) {
  if (n_act == 0) return cudaSuccess;
#define BKD_FIND_CASE(DIM)                                                  \
  case DIM:                                                                 \
    find_leaf_kernel<DIM><<<blocks(n_act, kFindThreads), kFindThreads, 0,   \
                            s>>>(t, qpad, act, n_act, n_act_dev, state,     \
                                 lst_d, K, placed, cnt);                    \
    return cudaGetLastError();
  switch (t.Dp) { BKD_DIMS(BKD_FIND_CASE) default: break; }
#undef BKD_FIND_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_bucket(const int2* placed, const uint32_t* act,
                          int n_act, int n_leaves, int tile,
                          const int32_t* leaf_cnt, const int32_t* cnt,
                          int32_t* off, int32_t* cursor, int32_t* toff,
                          Item* items, uint32_t* next, Counters* ctr,
                          cudaStream_t s, const int32_t* n_act_dev,
                          int32_t* n_next_dev) {
  // the cursor array (4 bytes per leaf) holds the 16-byte tile sums (one per
  // 2,048 leaves)
  ScanPart* parts = reinterpret_cast<ScanPart*>(cursor);
  const int nparts = blocks(n_leaves, kScanTile);
  scan_parts_kernel<<<nparts, kScanBlock, 0, s>>>(cnt, n_leaves, tile,
                                                  leaf_cnt, parts);
  scan_write_kernel<<<nparts, kScanBlock, 0, s>>>(cnt, n_leaves, tile,
                                                  leaf_cnt, parts, off, toff,
                                                  items, ctr, n_next_dev);
  if (n_act > 0)
    scatter_kernel<<<blocks(n_act, 256), 256, 0, s>>>(placed, act, n_act,
                                                      n_act_dev, off, next);
  return cudaGetLastError();
}

cudaError_t launch_chunk_items(const int32_t* toff, const int32_t* off,
                               const int32_t* leaf, int count,
                               int32_t* chunk_item, cudaStream_t s) {
  chunk_items_kernel<<<blocks(count, 128), 128, 0, s>>>(toff, off, leaf,
                                                        count, chunk_item);
  return cudaGetLastError();
}

}  // namespace bkd
