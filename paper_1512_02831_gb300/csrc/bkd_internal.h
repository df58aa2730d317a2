// bkd_internal.h -- shared declarations of the buffer k-d tree library.
//
// Device data layout (HBM, or pinned host memory in chunked mode):
//   top tree   float split[2^h - 1], heap order (node v: children 2v+1, 2v+2;
//              level(v) = floor(log2(v+1)); split dimension = level mod d).
//   leaf structure "quads": slot s of the leaf structure belongs to leaf
//              s / Lcap (Lcap = largest leaf size rounded up to 4); groups of
//              four consecutive slots form a quad of Dp float4 (Dp >= d is the
//              compiled dimension), dimension-major inside the quad:
//                  coord(s, i) = pts[(s/4)*4*Dp + 4*i + s%4].
//              Slots past a leaf's size and dimensions past d hold +inf / 0,
//              so a padded slot scores +inf and a padded dimension adds an
//              exact zero.
//   orig       int64 orig[slot]: row of P at that slot, -1 for padding.
//   queries    float qpad[m * Dp], zero-padded rows.
//   k-best     float lst_d[m * K], uint32 lst_i[m * K] (K = k + 1 entries,
//              ascending, lst_d[q*K + K-1] is the pruning bound); slots.
//   boxes      float box[(2^(h+1) - 1) * 2Dp]: tight bounding box of the
//              points under each heap node (min row, then max row, each
//              Dp floats; padding dimensions hold [0, 0]).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

struct bkd_tree;

namespace bkd {

constexpr int kPipeTile = 64;     // queries per ProcessAllBuffers work item
constexpr int kStart = -1;        // traversal state: root not yet entered
constexpr int kDone = -2;         // traversal state: root reached twice
constexpr uint32_t kNoSlot = 0xffffffffu;

// Compiled dimensions of the leaf kernel and compiled list capacities.
constexpr int kDims[] = {2, 4, 6, 8, 10, 12, 16, 24, 32};
// X(Dp) for every entry of kDims (kernel instantiation lists).
#define BKD_DIMS(X) X(2) X(4) X(6) X(8) X(10) X(12) X(16) X(24) X(32)
constexpr int kCaps[] = {2, 4, 8, 12, 16, 32, 64};

int padded_dim(int d);       // smallest compiled dimension >= d (0: none)
int list_capacity(int K);    // smallest compiled capacity >= K (0: none)

// One unit of ProcessAllBuffers work: up to kPipeTile buffered queries
// (positions [start, start+count) of the bucketed active list) against
// every point of one leaf.
struct Item {
  int32_t leaf;
  int32_t start;
  int32_t count;
  int32_t pad;
};

// Device-side round counters, copied to the host once per round.
// Traversal state of one query between rounds: the heap index of its last
// (or pending) leaf, or kStart / kDone, in the low 32 bits; in the high 32
// bits the mask of path levels whose off-path child is finished (see
// traverse.cuh).
__host__ __device__ inline uint64_t trav_state(int node, uint32_t mask) {
  return ((uint64_t)mask << 32) | (uint32_t)node;
}
__host__ __device__ inline int state_node(uint64_t s) {
  return (int)(uint32_t)s;
}
__host__ __device__ inline uint32_t state_mask(uint64_t s) {
  return (uint32_t)(s >> 32);
}

struct Counters {
  int32_t n_next;           // queries bucketed into some leaf this round
  int32_t n_items;          // work items this round
  unsigned long long pairs; // (query, point) pairs the round scores
  int32_t n_fallback;       // queries sent to the binary64 search
  int32_t n_resorted;       // queries re-ordered by binary64 distances
  int32_t err;              // device-detected input errors (bit mask)
  int32_t screen_next;      // next work item of the running screen launch
  int32_t screen_ovf_items; // screen items handed to the float32 kernel
  int32_t n_items_kept;     // servers with deferral: items processed
  unsigned long long tail_pairs;   // (query, point) pairs of the tail kernel
  unsigned long long tail_visits;  // (query, leaf) visits of the tail kernel
  unsigned long long screen_kept;  // pairs the BF16 screen passed on
  unsigned long long leaf_pairs;   // (query, point) pairs the float32 leaf
                                   // kernel scored
  unsigned long long screen_bytes; // operand-tile bytes the screen streamed
  // sums over the rounds of a LazySearch (written by the bucketing)
  unsigned long long rounds_pairs;   // (query, point) pairs scheduled
  unsigned long long rounds_visits;  // (query, leaf) pairs bucketed
  unsigned long long rounds_items;   // work items
  unsigned long long rounds_run;     // rounds with at least one query
  unsigned long long screen_queued;  // pairs queued for exact rescoring
  unsigned long long screen_overflow;  // screen items whose queue overflowed
  unsigned long long leaf_bytes;  // leaf-structure bytes the float32 leaf
                                  // kernel staged (one pass per work item)
  unsigned long long fallback_points;  // points the binary64 fallback
                                       // search scanned
  unsigned long long tail_mapped_pairs;  // tail pairs read from mapped
                                         // host memory (chunked trees)
};

constexpr int kErrNonFinite = 1;   // a query holds a non-finite / huge value
constexpr int kErrBadList = 2;     // a finished list holds an empty entry
constexpr int kErrTimeout = 4;     // a bounded device-side wait ran out

// Everything the kernels need about the tree.
struct DevTree {
  const float* split;      // 2^h - 1 (device)
  const float* pts;        // quads (device in resident mode, mapped host in
                           // chunked mode; used by the binary64 checks)
  const int64_t* orig;     // slot -> original index (device or mapped host)
  const int32_t* leaf_cnt; // points per leaf (device)
  const float* box;        // per-node bounding boxes, 2Dp floats each (device)
  int64_t n;
  int d, Dp, h;
  int64_t lcap;            // slots per leaf (multiple of 4)
  // chunked mode: N leaf chunks (chunk of leaf l = floor(l N / 2^h)) and,
  // per chunk, whether the last round scanned its buffers (device; nullptr
  // in resident mode, where every round scans every buffer)
  int n_chunks;
  const uint8_t* chunk_done;
  // servers with buffer deferral: per query slot, 1 while the query's
  // pending leaf was left unscanned (its buffer deferred); FindLeafBatch then
  // keeps it there (nullptr: every round scans every buffer)
  const uint8_t* q_wait = nullptr;
};

// ------------------------------------------------------------- launchers
// Queries Q (m x d, device) padded into qpad, lists +inf, state "start",
// act[q] = act_base + q (the slot numbers of the queries); non-finite or
// huge inputs set kErrNonFinite in ctr->err.
cudaError_t launch_init(const float* Q, int64_t m, int d, int Dp, float* qpad,
                        float* lst_d, uint32_t* lst_i, int K, uint64_t* state,
                        uint32_t* act, uint32_t act_base, Counters* ctr,
                        cudaStream_t s);

// Continuous batching helpers (serve.cu): v[0..n) = value; for every
// position of `act` whose query finished (placed.x < 0) one less in
// batch_left[slot_batch[slot]].
cudaError_t launch_fill(int32_t* v, int64_t n, int32_t value, cudaStream_t s);
cudaError_t launch_retire(const int2* placed, const uint32_t* act, int n_act,
                          const int32_t* slot_batch, int32_t* batch_left,
                          cudaStream_t s);
// ... and for every query of act[0..n) (all finished).
cudaError_t launch_retire_list(const uint32_t* act, int n,
                               const int32_t* slot_batch, int32_t* batch_left,
                               cudaStream_t s);

// FindLeafBatch from the traversal states in `state` (kStart for the first
// round): per position of `act`, placed = (next leaf, rank among the
// queries that go to it) or (-1, 0) when done; the new pending leaf in
// state; cnt[leaf] counts the queries that go on (cnt must start at 0).
// In chunked mode a query whose pending leaf lies in a chunk the last round
// did not scan (t.chunk_done) stays in that leaf's buffer: it is placed
// there again and its traversal does not advance.
// n_act_dev (optional): the active count read on the device (rounds queued
// without a host round trip); n_act is then an upper bound (grid size).
cudaError_t launch_find_leaf(const DevTree& t, const float* qpad,
                             const uint32_t* act, int n_act, uint64_t* state,
                             const float* lst_d, int K, int2* placed,
                             int32_t* cnt, cudaStream_t s,
                             const int32_t* n_act_dev = nullptr);

// Buffer insertion from per-leaf counts `cnt` and the placements of
// FindLeafBatch: offsets, work items of `tile` queries, round totals, and
// the active list bucketed by leaf into `next`.  cursor must hold
// max(n_leaves, 4) int32: between the two scan passes it carries one
// 16-byte partial sum per 2,048 leaves.
// n_act_dev as in launch_find_leaf; n_next_dev (optional) receives the
// round's bucketed count (the next round's active count).
cudaError_t launch_bucket(const int2* placed, const uint32_t* act,
                          int n_act, int n_leaves, int tile,
                          const int32_t* leaf_cnt, const int32_t* cnt,
                          int32_t* off, int32_t* cursor, int32_t* toff,
                          Item* items, uint32_t* next, Counters* ctr,
                          cudaStream_t s, const int32_t* n_act_dev = nullptr,
                          int32_t* n_next_dev = nullptr);

// For the leaves leaf[0..count): chunk_item[i] = the first work item of
// leaf[i] and chunk_item[count + i] = its first buffered query (leaf bounds
// of the chunks -> their item and query ranges).
cudaError_t launch_chunk_items(const int32_t* toff, const int32_t* off,
                               const int32_t* leaf, int count,
                               int32_t* chunk_item, cudaStream_t s);

// The part of each leaf a leaf-kernel launch scans: every point (leaf_lo
// nullptr), or the leaf-structure positions [pos_lo, pos_hi) of a
// point-split chunk (leaf_lo: 2^h + 1 leaf bounds on the device).
struct LeafPart {
  const int64_t* leaf_lo = nullptr;
  int64_t pos_lo = 0, pos_hi = 0;
};

// ProcessAllBuffers over items [item_lo, item_hi) (item_hi < 0: read the
// count on the device, from count_dev if given, else ctr->n_items).  pts /
// leaf0: the quads of leaf `leaf0` start at pts.
cudaError_t launch_leaf(const DevTree& t, int cap, const Item* items,
                        int item_lo, int item_hi, Counters* ctr,
                        const float* pts, int64_t leaf0, const uint32_t* act,
                        const float* qpad, float* lst_d, uint32_t* lst_i,
                        int K, int grid, cudaStream_t s,
                        const int32_t* count_dev = nullptr,
                        LeafPart part = LeafPart());

int leaf_kernel_grid(int Dp, int cap, int sm_count);

// BF16 screen data on the device.  Two screen kernels, each with the point
// operands in its own layout (either may be absent): the warp kernel
// (mma.sync fragments, fill_screen_warp; kind 0) and the tcgen05 kernel
// (128-row operand tiles, fill_screen; kind 1).  `kind` selects the kernel
// that runs; the centre, bmax and pnmax arrays serve both.
struct ScreenData {
  const uint16_t* words = nullptr;  // tcgen05: operand tiles, `tiles` per leaf
  const uint32_t* wwords = nullptr;  // warp kernel: fragments, `stride` slots
  const float* center = nullptr;
  const float* bmax = nullptr;
  const float* pnmax = nullptr;
  int64_t tiles = 0;   // tcgen05: 128-point tiles per leaf
  int64_t stride = 0;  // warp kernel: slots per leaf
  int kh = 0;          // tcgen05: k-halves (screen_halves)
  int wkh = 0;         // warp kernel: k-halves (screen_halves_warp)
  int kind = 0;
  // first leaf held by wwords (chunked trees: the chunk in a device chunk
  // buffer; its points are then at DevTree::pts from slot leaf0 * lcap on)
  int64_t leaf0 = 0;
  bool has(int k) const { return k == 0 ? wwords != nullptr : words != nullptr; }
  bool on() const { return has(kind); }
};
// Queries per work item of a screened round, by kernel (the warp kernel:
// one query column per lane; tcgen05: the MMA's N <= 128).
constexpr int kWarpScreenTile = 32;
inline int screen_tile_of(int kind) { return kind == 0 ? kWarpScreenTile : 128; }
// Slots per leaf of the warp kernel's arrays: the leaf capacity rounded up
// to its 32-point super-tile (two 16-point m-tiles).
inline int64_t screen_stride(int64_t lcap) { return (lcap + 31) / 32 * 32; }

// The screen's tensor-core shape: points are the MMA's M = 128 rows (one
// operand tile of a leaf), the buffered queries of one leaf its N <= 128
// columns (one work item), K = 16 slots per k-half.
constexpr int kScreenRows = 128;
constexpr int kScreenTile = 128;  // tcgen05: queries per work item
inline int64_t screen_tiles(int64_t lcap) {
  return (lcap + kScreenRows - 1) / kScreenRows;
}
// Byte offset of row r's k-group kg (slots 8 kg .. 8 kg + 7) in an operand
// tile of kh k-halves: the canonical no-swizzle K-major layout of the MMA
// (8-row core matrices of 16-byte rows; core matrices adjacent in K 128
// bytes apart, 8-row groups 256 kh bytes apart).
__host__ __device__ inline uint32_t screen_row_offset(int r, int kg, int kh) {
  return (uint32_t)((r >> 3) * (256 * kh) + kg * 128 + (r & 7) * 16);
}

// Workspace of the screened rounds, sized for the most work items a round
// can have: per item its query operand tile (128 x 32 kh bytes), a segment
// of screen_seg_cap() survivor entries and screen_cnt_per_item() counts
// (one per sub-segment), and room for the items handed to the float32
// kernel.
struct ScreenWork {
  uint8_t* bop = nullptr;
  uint32_t* seg = nullptr;
  int32_t* seg_cnt = nullptr;
  Item* ovf = nullptr;
};
int64_t screen_seg_cap();
int64_t screen_cnt_per_item();

// ProcessAllBuffers with the BF16 tensor-core screen and exact float32
// rescoring; same candidate lists as launch_leaf on a resident tree, over
// the round's items of at most screen_tile_of(sd.kind) queries (n_items <
// 0: the count is read on the device), by the kernel sd.kind selects:
//   kind 0 (k_screen_warp.cu): one warp per item, mma.sync, survivors
//     rescored by the same warp (ScreenWork, cap and leaf_grid unused);
//   kind 1 (k_screen.cu): three kernels: the items' query operands, the
//     tcgen05 screen (survivors to per-item segments), the exact
//     rescoring; items whose segment overflowed go to the float32 leaf
//     kernel (capacity `cap`, grid leaf_grid).
// screen_grid: resident CTAs of the selected kernel (0 if it does not fit:
// shared memory, tensor memory, leaf capacity).
int screen_grid(const ScreenData& sd, int Dp, int64_t lcap, int K,
                int sm_count);
cudaError_t launch_screen(const DevTree& t, const ScreenData& sd,
                          const Item* items, int n_items, Counters* ctr,
                          const uint32_t* act, const float* qpad,
                          float* lst_d, uint32_t* lst_i, int K, int grid,
                          const ScreenWork& w, int cap, int leaf_grid,
                          int sm_count, cudaStream_t s);
// The warp kernel (k_screen_warp.cu), items [item_lo, item_hi) (item_hi <
// 0: the device's count of the round).
int screen_grid_warp(int kh, int64_t lcap, int K, int sm_count);
cudaError_t launch_screen_warp(const DevTree& t, const ScreenData& sd,
                               const Item* items, int item_lo, int item_hi,
                               Counters* ctr, const uint32_t* act,
                               const float* qpad, float* lst_d,
                               uint32_t* lst_i, int K, int grid,
                               cudaStream_t s);

// Runs the traversal of each of the n_act queries in `act` to its end (one
// warp per query); state[q] is the query's pending (not yet scanned) leaf.
// `pts` is the leaf structure (device or mapped host).
// Leaves held in device chunk buffers (chunked trees): leaves [lo, hi) of
// buffer b start at buf[b] (empty range: none); other leaves are read at
// `pts` (mapped pinned host memory), counted in Counters::tail_mapped_pairs.
struct ChunkBufs {
  const float* buf[2] = {nullptr, nullptr};
  int64_t lo[2] = {0, 0}, hi[2] = {0, 0};
};
// (after_scanned: state[q] holds the leaf the query scanned last, not one
// still to scan: the walk starts at the leaf after it -- except for the
// queries whose t.q_wait flag is set: their pending leaf is still to scan)
cudaError_t launch_tail(const DevTree& t, const float* pts,
                        const uint32_t* act, int n_act, uint64_t* state,
                        const float* qpad, float* lst_d, uint32_t* lst_i,
                        int K, Counters* ctr, int sm_count, cudaStream_t s,
                        const ChunkBufs& cb = ChunkBufs(),
                        bool after_scanned = false);

cudaError_t launch_recheck(const DevTree& t, int64_t m, int k, int K,
                           const float* qpad, const float* lst_d,
                           const uint32_t* lst_i, int64_t* out_idx,
                           float* out_dist, uint32_t* fb_list, Counters* ctr,
                           cudaStream_t s);

// (ctr, if given: its fallback_points counts the points scanned)
cudaError_t launch_fallback(const DevTree& t, int n_fb, const uint32_t* fb_list,
                            int k, int K, const float* qpad, const float* lst_d,
                            int64_t* out_idx, float* out_dist, cudaStream_t s,
                            Counters* ctr = nullptr);

// Outlier score of Sec. 4.3 (k_outlier.cu): inv[orig[s]] = s for every
// occupied slot; Q[r] = the point of original index i0 + r (r < m), read
// from the quads at pts; out[r] = mean of the square roots of the k
// distances of row r of the (k+1)-lists idx / dist, without the point's own
// index (or without the last entry if the row does not hold it).
cudaError_t launch_inverse(const int64_t* orig, int64_t slots, int64_t* inv,
                           cudaStream_t s);
cudaError_t launch_gather(const float* pts, int Dp, int d, const int64_t* inv,
                          int64_t i0, int64_t m, float* Q, cudaStream_t s);
cudaError_t launch_score(const int64_t* idx, const float* dist, int64_t i0,
                         int64_t m, int k, float* out, cudaStream_t s);

// Read-only view of a tree handle for entry points outside api.cu.
struct TreeView {
  int device;
  int sm_count;
  cudaStream_t stream;
  DevTree dev;
  int64_t n_leaves;
  bool chunked;
  const float* d_pts;        // resident leaf structure (nullptr if chunked)
  Counters* h_ctr;           // pinned host counter block of the handle
  ScreenData screen;         // BF16 screen data (words == nullptr: none)
  int precision;             // current leaf-scoring option (0 / 1)
  int tail_queries;          // tail threshold option (-1: automatic)
  int rescue_rounds;         // server straggler rescue (0: never)
  int defer_queries;         // server buffer trigger (0: off)
};
TreeView view_of(const struct ::bkd_tree* t);

// Every device and pinned host allocation of the library goes through these
// two (api.cu): they count down the test hook of bkd_test_fail_alloc and
// report cudaErrorMemoryAllocation for the chosen allocation.
cudaError_t dev_malloc_raw(void** p, size_t bytes);
cudaError_t host_alloc_raw(void** p, size_t bytes, unsigned flags);
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}
template <class T>
inline cudaError_t host_alloc(T** p, size_t bytes, unsigned flags) {
  return host_alloc_raw(reinterpret_cast<void**>(p), bytes, flags);
}

// Records the calling thread's bkd_last_error() message; returns `code`.
int set_error(int code, const char* fmt, ...);

// Host tree construction (build.cpp).
struct HostTree {
  int64_t n = 0;
  int d = 0, Dp = 0, h = 0;
  int64_t lcap = 0;
  float* split = nullptr;     // 2^h - 1 (at least one element)
  int64_t* leaf_lo = nullptr; // 2^h + 1
  int64_t* perm = nullptr;    // n
};

// Builds split / leaf_lo / perm of the median-split tree over host P.
// Returns 0 or an error message (static string).
const char* build_host_tree(const float* P, int64_t n, int d, int h,
                            HostTree* out);

// Bounding box of the points under every heap node (2^(h+1) - 1 nodes):
// box[v*2Dp .. v*2Dp+Dp) = per-dimension minimum, box[v*2Dp+Dp .. v*2Dp+2Dp)
// = maximum; dimensions d..Dp-1 are [0, 0].
void fill_boxes(const float* P, const HostTree& t, float* box);

// k-halves of 16 bf16 slots the BF16 screen uses: the d offsets, two slots
// for the point's squared norm and three for the query's threshold (1 for
// d <= 11, 2 for d <= 27, else 3).
inline int screen_halves(int d) { return (d + 5 + 15) / 16; }
// The warp kernel's k-halves: the d offsets and the norm split (its
// threshold is compared in the epilogue): 1 for d <= 14, 2 for d <= 30,
// else 3.
inline int screen_halves_warp(int d) { return (d + 2 + 15) / 16; }

// Data of the BF16 screen, per leaf: the centre c (midpoint of the leaf's
// bounding box); per point (a row of the leaf's operand tiles, `tiles` of
// 128 rows each, 128 x 16 kh bf16 per tile in the layout of
// screen_row_offset) its offset bf16(fl(x - c)) in slots 0..d-1, its
// squared norm pn (binary64 sum rounded to float) split as pn_hi = bf16(pn),
// pn_lo = bf16(pn - pn_hi) in slots d, d+1, and 1.0 in slots d+2..d+4
// (padding rows: pn_hi = +inf, everything else 0); per leaf bmax (upper
// bound on the offset rounding error norm) and pnmax (largest pn, floored
// at 2^-86, so that the screens' error term 2^-14 (|v^|^2 + pnmax) holds an
// absolute 2^-100 that covers the errors of underflow).
void fill_screen(const float* P, const HostTree& t, int64_t tiles,
                 uint16_t* words, float* center, float* bmax, float* pnmax);
// The warp kernel's layout of the same per-point slots (offsets, pn_hi,
// pn_lo; no threshold slots): `stride` slots per leaf and k-half, 8 words
// (bf16 pairs) per point in m16n8k16 A-fragment order, grouped in 32-point
// super-tiles (lane (g, t) of a warp reads its two rows of both m-tiles of
// a k-half with one 16-byte load); padding points pn_hi = +inf.  Fills
// center, bmax and pnmax like fill_screen.
void fill_screen_warp(const float* P, const HostTree& t, int64_t stride,
                      uint32_t* words, float* center, float* bmax,
                      float* pnmax);

// Writes the quads and orig arrays for leaves [leaf_lo_id, leaf_hi_id)
// into host buffers (`pts` and `orig` point at leaf leaf_lo_id's first slot).
void fill_quads(const float* P, const HostTree& t, int64_t leaf_lo_id,
                int64_t leaf_hi_id, float* pts, int64_t* orig);

}  // namespace bkd
