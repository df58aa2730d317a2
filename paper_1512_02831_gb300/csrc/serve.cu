// serve.cu -- continuous batching over a resident tree (bkd_serve_*).
//
// The paper's querying phase fetches new queries from the input queue while
// earlier ones are still in flight (Algorithm 1; Sec. 3.2 on-the-fly
// querying).  Here that queue takes whole batches of any size and k:
//
//   admit     queued batches, first come first served, get contiguous query
//             slots while free slots fit them; their queries are padded into
//             the slots, their lists set to +inf, their traversal to "start",
//             and their slot numbers appended to the active list;
//   round     one LazySearch round over every active query, whatever its
//             batch: FindLeafBatch, buffer insertion, ProcessAllBuffers (the
//             same kernels as bkd_query);
//   complete  a batch whose queries have all finished gets the binary64
//             re-check and fallback and its results, and frees its slots.
//
// Batches are routed by k to one of up to three class servers (lists of at
// most 12, 32 or 64 entries), each a complete server of its own (slots,
// active list, rounds).  Every query of a class carries a list of the
// class's k_max + 1 entries.  After the rounds a query's list holds its
// k_max + 1 smallest float32 distances, so its first k + 1 entries are the
// k + 1 smallest: the re-check and fallback of a batch with k <= k_max see
// exactly what a bkd_query with that k sees, and the results are the same
// (both equal the binary64 definition).
//
// Queries admitted in a step take their first leaf in a round of their own
// on the float32 leaf kernel (their lists are still empty, so the BF16
// screen could reject nothing); the shared round of the step then follows
// the tree's precision option for everyone.
#include <cuda_runtime.h>

#include <algorithm>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "bkd.h"
#include "bkd_internal.h"
#include "slots.h"

using namespace bkd;

namespace {

constexpr int kMaxBatches = 4096;  // batches admitted at once

#define SV_CU(call)                                                        \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess)                                                 \
      return set_error(e_ == cudaErrorMemoryAllocation ? BKD_ENOMEM        \
                                                       : BKD_ECUDA,        \
                       "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

// 1: device memory the tree's GPU can use (its own, or managed); 0: host
// memory; -1: device memory of another GPU (refused: no peer access).
int device_ptr(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (a.type == cudaMemoryTypeManaged) return 1;
  if (a.type == cudaMemoryTypeDevice) return a.device == device ? 1 : -1;
  return 0;
}

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
      cudaSetDevice(prev);
  }
};

struct Batch {
  int64_t ticket = 0;
  const float* Q = nullptr;
  int64_t m = 0;
  int k = 0;
  int64_t* out_idx = nullptr;
  float* out_dist = nullptr;
  bool q_dev = false, o_dev = false;
  int64_t s0 = -1;  // first slot
  int bid = -1;     // index into batch_left
  int status = BKD_BATCH_QUEUED;
  int64_t born = 0;  // the class server's round count at admission
};

// A batch still running BKD_OPT_RESCUE_ROUNDS rounds after its admission
// has its remaining queries finished by the tail kernel (one warp per query,
// to the end of its traversal): a batch completes only with its last query,
// and the stragglers of a large batch would otherwise take hundreds of
// rounds more.

// Buffer trigger (BKD_OPT_DEFER_QUERIES): a leaf's buffer is processed in
// a round when it holds at least min_q queries or was deferred kDeferMax
// rounds in a row; go[l] says which, leaf_wait[l] counts the deferrals.
constexpr int kDeferMax = 4;

__global__ void defer_leaves_kernel(const int32_t* __restrict__ cnt,
                                    int64_t L, int min_q,
                                    int32_t* __restrict__ leaf_wait,
                                    uint8_t* __restrict__ go) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  const int c = cnt[l];
  if (c == 0) {
    leaf_wait[l] = 0;
    go[l] = 0;
    return;
  }
  const bool g = c >= min_q || leaf_wait[l] >= kDeferMax;
  go[l] = g ? 1 : 0;
  leaf_wait[l] = g ? 0 : leaf_wait[l] + 1;
}

// The round's work items of the leaves that go, to `out` (count in
// ctr->n_items_kept; order free); each item's queries get their wait flag:
// 0 (scanned this round) or 1 (the pending leaf stays to scan).
__global__ void filter_items_kernel(const Item* __restrict__ items,
                                    Counters* ctr,
                                    const uint8_t* __restrict__ go,
                                    const uint32_t* __restrict__ act,
                                    uint8_t* __restrict__ q_wait,
                                    Item* __restrict__ out) {
  const int n = ctr->n_items;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < n;
       it += gridDim.x * blockDim.x) {
    const Item w = items[it];
    const bool g = go[w.leaf] != 0;
    if (g) out[atomicAdd(&ctr->n_items_kept, 1)] = w;
    for (int j = 0; j < w.count; ++j) q_wait[act[w.start + j]] = g ? 0 : 1;
  }
}

__global__ void take_kept_items_kernel(Counters* ctr) {
  ctr->n_items = ctr->n_items_kept;
}

// Splits the active list by the rescue flag of each query's batch: young
// queries to `young`, those of batches to rescue to `old` (counts in
// cnt[0], cnt[1]; order within each list is free).
__global__ void partition_kernel(const uint32_t* __restrict__ act, int n,
                                 const int32_t* __restrict__ slot_batch,
                                 const uint8_t* __restrict__ rescue,
                                 uint32_t* __restrict__ young,
                                 uint32_t* __restrict__ old,
                                 int32_t* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t q = act[i];
  if (rescue[slot_batch[q]])
    old[atomicAdd(cnt + 1, 1)] = q;
  else
    young[atomicAdd(cnt, 1)] = q;
}

template <class T>
cudaError_t dev_alloc(T** p, int64_t n) {
  return dev_malloc(p, std::max<int64_t>(n, 1) * sizeof(T));
}

}  // namespace

struct ClassServer {
  bkd_tree* tree = nullptr;
  TreeView v{};  // refreshed every step (stream, precision option)
  int kmax = 0, K = 0, cap = 0;
  int64_t max_q = 0;
  int grid_max = 0, screen_max = 0;
  // per slot
  float *qstage = nullptr, *qpad = nullptr, *lst_d = nullptr;
  uint32_t *lst_i = nullptr, *act_a = nullptr, *act_b = nullptr,
           *fb = nullptr;
  uint64_t* state = nullptr;
  int2* placed = nullptr;
  int32_t* slot_batch = nullptr;
  int64_t* out_i = nullptr;
  float* out_d = nullptr;
  // per leaf / per round
  int32_t *cnt = nullptr, *off = nullptr, *cursor = nullptr, *toff = nullptr;
  Item* items = nullptr;
  ScreenWork sw;            // screened rounds' workspace (see ScreenWork)
  int32_t* batch_left = nullptr;  // device, kMaxBatches
  Counters *d_ctr = nullptr, *d_fin = nullptr;
  Counters *h_ctr = nullptr, *h_fin = nullptr;  // pinned
  int32_t* h_left = nullptr;                    // pinned, kMaxBatches
  // straggler rescue
  int64_t rounds = 0;            // rounds run
  uint8_t* d_rescue = nullptr;   // device, kMaxBatches flags
  uint8_t* h_rescue = nullptr;   // pinned, kMaxBatches
  uint32_t* resc = nullptr;      // device, queries to rescue
  int32_t* d_part = nullptr;     // device, 2 counts
  int32_t* h_part = nullptr;     // pinned, 2 counts
  // buffer trigger
  uint8_t* q_wait = nullptr;     // device, per slot
  int32_t* leaf_wait = nullptr;  // device, per leaf
  uint8_t* leaf_go = nullptr;    // device, per leaf
  Item* items2 = nullptr;        // device, the items processed in a round
  bool waiting = false;          // some q_wait flag may be set
  // the tree with this server's wait flags (while any may be set)
  DevTree dev() const {
    DevTree D = v.dev;
    if (waiting) D.q_wait = q_wait;
    return D;
  }
  // host state
  uint32_t* act = nullptr;
  uint32_t* nxt = nullptr;
  int n_act = 0;
  Slots slots;
  std::vector<int> free_bids;
  std::deque<Batch*> queue;
  std::vector<Batch*> running;  // by batch id
  std::map<int64_t, std::unique_ptr<Batch>> batches;
  int64_t next_ticket = 1;

  ~ClassServer() {
    cudaFree(qstage);
    cudaFree(qpad);
    cudaFree(lst_d);
    cudaFree(lst_i);
    cudaFree(act_a);
    cudaFree(act_b);
    cudaFree(fb);
    cudaFree(state);
    cudaFree(placed);
    cudaFree(slot_batch);
    cudaFree(out_i);
    cudaFree(out_d);
    cudaFree(cnt);
    cudaFree(off);
    cudaFree(cursor);
    cudaFree(toff);
    cudaFree(items);
    cudaFree(sw.bop);
    cudaFree(sw.seg);
    cudaFree(sw.seg_cnt);
    cudaFree(sw.ovf);
    cudaFree(batch_left);
    cudaFree(d_ctr);
    cudaFree(d_fin);
    cudaFreeHost(h_ctr);
    cudaFreeHost(h_fin);
    cudaFreeHost(h_left);
    cudaFree(d_rescue);
    cudaFree(resc);
    cudaFree(d_part);
    cudaFreeHost(h_rescue);
    cudaFreeHost(h_part);
    cudaFree(q_wait);
    cudaFree(leaf_wait);
    cudaFree(leaf_go);
    cudaFree(items2);
  }

  void finish(Batch* b, int status) {
    b->status = status;
    if (b->s0 >= 0) slots.give(b->s0, b->m);
    if (b->bid >= 0) {
      running[b->bid] = nullptr;
      free_bids.push_back(b->bid);
    }
    b->s0 = -1;
    b->bid = -1;
  }

  int admit(Batch* b, int64_t s0, int bid, bool* ok);
  int complete(Batch* b);
  int first_round(int n_old);
  int rescue();
  int round();
};

// Copies a batch's queries into its slots and appends them to the active
// list; a non-finite query fails the batch (ok = false).
int ClassServer::admit(Batch* b, int64_t s0, int bid, bool* ok) {
  const DevTree& D = v.dev;
  cudaStream_t s = v.stream;
  const int64_t m = b->m;
  SV_CU(cudaMemcpyAsync(qstage + s0 * D.d, b->Q, sizeof(float) * m * D.d,
                        b->q_dev ? cudaMemcpyDeviceToDevice
                                 : cudaMemcpyHostToDevice,
                        s));
  SV_CU(cudaMemsetAsync(d_fin, 0, sizeof(Counters), s));
  SV_CU(launch_init(qstage + s0 * D.d, m, D.d, D.Dp, qpad + s0 * D.Dp,
                    lst_d + s0 * K, lst_i + s0 * K, K, state + s0,
                    act + n_act, (uint32_t)s0, d_fin, s));
  SV_CU(launch_fill(slot_batch + s0, m, bid, s));
  SV_CU(launch_fill(batch_left + bid, 1, (int32_t)m, s));
  SV_CU(cudaMemsetAsync(q_wait + s0, 0, m, s));
  SV_CU(cudaMemcpyAsync(h_fin, d_fin, sizeof(Counters),
                        cudaMemcpyDeviceToHost, s));
  SV_CU(cudaStreamSynchronize(s));
  *ok = !(h_fin->err & kErrNonFinite);
  return BKD_OK;
}

// The first leaf of the queries admitted in this step (active positions
// [n_old, n_act)): FindLeafBatch, bucketing and the float32 leaf kernel over
// them alone.  Their processed list goes to the scratch `nxt`; they stay in
// the active list for the shared round.
int ClassServer::first_round(int n_old) {
  const DevTree& D = v.dev;
  cudaStream_t s = v.stream;
  const int64_t L = v.n_leaves;
  const int n_new = n_act - n_old;
  SV_CU(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * L, s));
  SV_CU(launch_find_leaf(D, qpad, act + n_old, n_new, state, lst_d, K,
                         placed + n_old, cnt, s));
  SV_CU(launch_retire(placed + n_old, act + n_old, n_new, slot_batch,
                      batch_left, s));
  SV_CU(launch_bucket(placed + n_old, act + n_old, n_new, (int)L, kPipeTile,
                      D.leaf_cnt, cnt, off, cursor, toff, items, nxt, d_ctr,
                      s));
  SV_CU(cudaMemcpyAsync(h_ctr, d_ctr, sizeof(Counters),
                        cudaMemcpyDeviceToHost, s));
  SV_CU(cudaStreamSynchronize(s));
  if (h_ctr->n_next > 0)
    SV_CU(launch_leaf(D, cap, items, 0, h_ctr->n_items, d_ctr, v.d_pts, 0,
                      nxt, qpad, lst_d, lst_i, K,
                      std::min(grid_max, h_ctr->n_items), s));
  return BKD_OK;
}

// The queries of batches admitted BKD_OPT_RESCUE_ROUNDS rounds ago or
// earlier leave the active list and are finished by the tail kernel (their
// state holds the leaf they scanned last).
int ClassServer::rescue() {
  const int64_t after = v.rescue_rounds;
  if (after <= 0) return BKD_OK;
  const DevTree D = dev();  // a deferred query's pending leaf is unscanned
  bool any = false;
  for (int bid = 0; bid < kMaxBatches; ++bid) {
    const Batch* b = running[bid];
    h_rescue[bid] = b && rounds - b->born >= after;
    any = any || h_rescue[bid];
  }
  if (!any || n_act == 0) return BKD_OK;
  cudaStream_t s = v.stream;
  SV_CU(cudaMemcpyAsync(d_rescue, h_rescue, kMaxBatches,
                        cudaMemcpyHostToDevice, s));
  SV_CU(cudaMemsetAsync(d_part, 0, 2 * sizeof(int32_t), s));
  partition_kernel<<<(n_act + 255) / 256, 256, 0, s>>>(act, n_act, slot_batch,
                                                       d_rescue, nxt, resc,
                                                       d_part);
  SV_CU(cudaGetLastError());
  SV_CU(cudaMemcpyAsync(h_part, d_part, 2 * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, s));
  SV_CU(cudaStreamSynchronize(s));
  const int n_young = h_part[0], n_old = h_part[1];
  if (n_old > 0) {
    SV_CU(launch_tail(D, v.d_pts, resc, n_old, state, qpad, lst_d, lst_i, K,
                      d_ctr, v.sm_count, s, ChunkBufs(), true));
    SV_CU(launch_retire_list(resc, n_old, slot_batch, batch_left, s));
  }
  std::swap(act, nxt);
  n_act = n_young;
  return BKD_OK;
}

// One LazySearch round over the whole active list.
int ClassServer::round() {
  const DevTree D = dev();
  cudaStream_t s = v.stream;
  const int64_t L = v.n_leaves;
  const bool screened = v.precision == 1 && screen_max > 0;
  SV_CU(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * L, s));
  SV_CU(launch_find_leaf(D, qpad, act, n_act, state, lst_d, K, placed, cnt,
                         s));
  SV_CU(launch_retire(placed, act, n_act, slot_batch, batch_left, s));
  SV_CU(launch_bucket(placed, act, n_act, (int)L,
                      screened ? screen_tile_of(v.screen.kind) : kPipeTile,
                      D.leaf_cnt, cnt, off,
                      cursor, toff, items, nxt, d_ctr, s));
  SV_CU(cudaMemcpyAsync(h_ctr, d_ctr, sizeof(Counters),
                        cudaMemcpyDeviceToHost, s));
  SV_CU(cudaMemcpyAsync(h_left, batch_left, sizeof(int32_t) * kMaxBatches,
                        cudaMemcpyDeviceToHost, s));
  SV_CU(cudaStreamSynchronize(s));
  if (h_ctr->err & kErrTimeout)
    return set_error(BKD_ETIMEOUT, "a leaf-segment copy did not complete");
  const int n_next = h_ctr->n_next, n_items = h_ctr->n_items;
  // few queries left in flight: the tail kernel finishes all of them now
  const int tail = v.tail_queries >= 0 ? v.tail_queries : 8192;
  if (n_next > 0 && n_next <= tail) {
    SV_CU(launch_tail(D, v.d_pts, nxt, n_next, state, qpad, lst_d, lst_i, K,
                      d_ctr, v.sm_count, s));
    SV_CU(launch_retire_list(nxt, n_next, slot_batch, batch_left, s));
    SV_CU(cudaMemcpyAsync(h_left, batch_left, sizeof(int32_t) * kMaxBatches,
                          cudaMemcpyDeviceToHost, s));
    SV_CU(cudaStreamSynchronize(s));
    n_act = 0;
    return BKD_OK;
  }
  if (n_next > 0) {
    // the buffer trigger: only the leaves that go are processed (the item
    // count is then read on the device); with the trigger off, one pass with
    // every leaf going clears flags a previous setting left
    const Item* its = items;
    int nit = n_items;
    if (v.defer_queries > 0 || waiting) {
      const int min_q = std::max(v.defer_queries, 1);
      SV_CU(cudaMemsetAsync(&d_ctr->n_items_kept, 0, sizeof(int32_t), s));
      defer_leaves_kernel<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(
          cnt, L, min_q, leaf_wait, leaf_go);
      filter_items_kernel<<<std::max(1, std::min((n_items + 255) / 256,
                                                 v.sm_count * 8)),
                            256, 0, s>>>(items, d_ctr, leaf_go, nxt, q_wait,
                                         items2);
      take_kept_items_kernel<<<1, 1, 0, s>>>(d_ctr);
      SV_CU(cudaGetLastError());
      its = items2;
      nit = -1;
      waiting = v.defer_queries > 0;
    }
    if (screened)
      SV_CU(launch_screen(D, v.screen, its, nit, d_ctr, nxt, qpad, lst_d,
                          lst_i, K, screen_max, sw, cap, grid_max,
                          v.sm_count, s));
    else
      SV_CU(launch_leaf(D, cap, its, 0, nit, d_ctr, v.d_pts, 0, nxt, qpad,
                        lst_d, lst_i, K,
                        nit >= 0 ? std::min(grid_max, nit) : grid_max, s));
  }
  std::swap(act, nxt);
  n_act = n_next;
  ++rounds;
  return BKD_OK;
}

// Re-check, fallback and results of a batch whose queries all finished.
int ClassServer::complete(Batch* b) {
  const DevTree& D = v.dev;
  cudaStream_t s = v.stream;
  const int64_t s0 = b->s0, m = b->m;
  const int k = b->k;
  int64_t* oi = b->o_dev ? b->out_idx : out_i + s0 * kmax;
  float* od = b->o_dev ? b->out_dist : out_d + s0 * kmax;
  SV_CU(cudaMemsetAsync(d_fin, 0, sizeof(Counters), s));
  SV_CU(launch_recheck(D, m, k, K, qpad + s0 * D.Dp, lst_d + s0 * K,
                       lst_i + s0 * K, oi, od, fb + s0, d_fin, s));
  SV_CU(cudaMemcpyAsync(h_fin, d_fin, sizeof(Counters),
                        cudaMemcpyDeviceToHost, s));
  SV_CU(cudaStreamSynchronize(s));
  if (h_fin->err & kErrBadList)
    return set_error(BKD_ECUDA, "internal error: a finished candidate list "
                                "holds an empty entry");
  if (h_fin->n_fallback > 0)
    SV_CU(launch_fallback(D, h_fin->n_fallback, fb + s0, k, K,
                          qpad + s0 * D.Dp, lst_d + s0 * K, oi, od, s));
  if (!b->o_dev) {
    SV_CU(cudaMemcpyAsync(b->out_idx, oi, sizeof(int64_t) * m * k,
                          cudaMemcpyDeviceToHost, s));
    SV_CU(cudaMemcpyAsync(b->out_dist, od, sizeof(float) * m * k,
                          cudaMemcpyDeviceToHost, s));
  }
  SV_CU(cudaStreamSynchronize(s));
  finish(b, BKD_BATCH_DONE);
  return BKD_OK;
}

namespace {

// A server of one list-capacity class (every query carries k_max + 1
// list entries).
int cs_open(bkd_tree* t, int k_max, int64_t max_queries, ClassServer** out) {
  *out = nullptr;
  const TreeView v = view_of(t);
  if (v.chunked)
    return set_error(BKD_EUNSUPPORTED,
                     "serving needs a tree resident in device memory");
  if (k_max < 1 || k_max > v.dev.n)
    return set_error(BKD_EINVAL, "k_max must be in [1, n] (got %d)", k_max);
  if (k_max > BKD_MAX_K)
    return set_error(BKD_EUNSUPPORTED, "k_max = %d exceeds BKD_MAX_K = %d",
                     k_max, BKD_MAX_K);
  if (max_queries < 1 || max_queries >= ((int64_t)1 << 31))
    return set_error(BKD_EINVAL, "max_queries must be in [1, 2^31)");
  DeviceScope guard(v.device);
  auto sv = std::make_unique<ClassServer>();
  sv->tree = t;
  sv->v = v;
  sv->kmax = k_max;
  sv->K = k_max + 1;
  sv->cap = list_capacity(sv->K);
  sv->max_q = max_queries;
  const int64_t Q = max_queries, L = v.n_leaves;
  const DevTree& D = v.dev;
  SV_CU(dev_alloc(&sv->qstage, Q * D.d));
  SV_CU(dev_alloc(&sv->qpad, Q * D.Dp));
  SV_CU(dev_alloc(&sv->lst_d, Q * sv->K));
  SV_CU(dev_alloc(&sv->lst_i, Q * sv->K));
  SV_CU(dev_alloc(&sv->act_a, Q));
  SV_CU(dev_alloc(&sv->act_b, Q));
  SV_CU(dev_alloc(&sv->fb, Q));
  SV_CU(dev_alloc(&sv->state, Q));
  SV_CU(dev_alloc(&sv->placed, Q));
  SV_CU(dev_alloc(&sv->slot_batch, Q));
  SV_CU(dev_alloc(&sv->out_i, Q * k_max));
  SV_CU(dev_alloc(&sv->out_d, Q * k_max));
  SV_CU(dev_alloc(&sv->cnt, L));
  SV_CU(dev_alloc(&sv->off, L + 1));
  SV_CU(dev_alloc(&sv->cursor, std::max<int64_t>(L, 4)));
  SV_CU(dev_alloc(&sv->toff, L + 1));
  SV_CU(dev_alloc(&sv->items, Q / std::min(kWarpScreenTile, kPipeTile) + L + 1));
  SV_CU(dev_alloc(&sv->batch_left, kMaxBatches));
  SV_CU(dev_alloc(&sv->d_ctr, 1));
  SV_CU(dev_alloc(&sv->d_fin, 1));
  SV_CU(host_alloc(&sv->h_ctr, sizeof(Counters), cudaHostAllocDefault));
  SV_CU(host_alloc(&sv->h_fin, sizeof(Counters), cudaHostAllocDefault));
  SV_CU(host_alloc(&sv->h_left, sizeof(int32_t) * kMaxBatches,
                      cudaHostAllocDefault));
  SV_CU(dev_alloc(&sv->q_wait, Q));
  SV_CU(dev_alloc(&sv->leaf_wait, L));
  SV_CU(dev_alloc(&sv->leaf_go, L));
  SV_CU(dev_alloc(&sv->items2, Q / std::min(kWarpScreenTile, kPipeTile) + L + 1));
  SV_CU(cudaMemsetAsync(sv->q_wait, 0, std::max<int64_t>(Q, 1), v.stream));
  SV_CU(cudaMemsetAsync(sv->leaf_wait, 0, sizeof(int32_t) * std::max<int64_t>(L, 1),
                        v.stream));
  SV_CU(dev_alloc(&sv->d_rescue, kMaxBatches));
  SV_CU(dev_alloc(&sv->resc, Q));
  SV_CU(dev_alloc(&sv->d_part, 2));
  SV_CU(host_alloc(&sv->h_rescue, kMaxBatches, cudaHostAllocDefault));
  SV_CU(host_alloc(&sv->h_part, 2 * sizeof(int32_t), cudaHostAllocDefault));
  SV_CU(cudaMemsetAsync(sv->d_ctr, 0, sizeof(Counters), v.stream));
  SV_CU(cudaMemsetAsync(sv->batch_left, 0, sizeof(int32_t) * kMaxBatches,
                        v.stream));
  SV_CU(cudaStreamSynchronize(v.stream));
  sv->grid_max = leaf_kernel_grid(D.Dp, sv->cap, v.sm_count);
  if (v.screen.on() && v.screen.kind == 1) {
    const int64_t si = Q / kScreenTile + L + 1;
    SV_CU(dev_alloc(&sv->sw.bop, si * 4096 * v.screen.kh));
    SV_CU(dev_alloc(&sv->sw.seg, si * screen_seg_cap()));
    SV_CU(dev_alloc(&sv->sw.seg_cnt, si * screen_cnt_per_item()));
    SV_CU(dev_alloc(&sv->sw.ovf, 2 * si));
  }
  sv->screen_max = v.screen.on()
                       ? screen_grid(v.screen, D.Dp, D.lcap, sv->K,
                                     v.sm_count)
                       : 0;
  if (sv->grid_max <= 0)
    return set_error(BKD_EUNSUPPORTED, "no leaf kernel for d = %d, k = %d",
                     D.d, k_max);
  sv->act = sv->act_a;
  sv->nxt = sv->act_b;
  sv->slots.reset(Q);
  sv->running.assign(kMaxBatches, nullptr);
  for (int i = kMaxBatches - 1; i >= 0; --i) sv->free_bids.push_back(i);
  *out = sv.release();
  return BKD_OK;
}

int cs_submit(ClassServer* s, const float* Q, int64_t m, int k,
              int64_t* out_idx, float* out_dist, int64_t* ticket) {
  if (m < 0 || m > s->max_q)
    return set_error(BKD_EINVAL, "m = %lld outside [0, max_queries = %lld]",
                     (long long)m, (long long)s->max_q);
  if (k < 1 || k > s->kmax)
    return set_error(BKD_EINVAL, "k = %d outside [1, k_max = %d]", k,
                     s->kmax);
  if (m > 0 && (!Q || !out_idx || !out_dist))
    return set_error(BKD_EINVAL, "Q / out_idx / out_dist is NULL");
  DeviceScope guard(s->v.device);
  const int qk = m > 0 ? device_ptr(Q, s->v.device) : 0;
  const int ik = m > 0 ? device_ptr(out_idx, s->v.device) : 0;
  const int dk = m > 0 ? device_ptr(out_dist, s->v.device) : 0;
  if (qk < 0 || ik < 0 || dk < 0)
    return set_error(BKD_EINVAL, "Q / out_idx / out_dist is device memory of "
                                 "another GPU than the tree's (device %d)",
                     s->v.device);
  auto b = std::make_unique<Batch>();
  b->ticket = s->next_ticket++;
  b->Q = Q;
  b->m = m;
  b->k = k;
  b->out_idx = out_idx;
  b->out_dist = out_dist;
  if (m > 0) {
    b->q_dev = qk == 1;
    b->o_dev = ik == 1 && dk == 1;
    s->queue.push_back(b.get());
  } else {
    b->status = BKD_BATCH_DONE;
  }
  *ticket = b->ticket;
  s->batches[b->ticket] = std::move(b);
  return BKD_OK;
}

int cs_step(ClassServer* s, int64_t* pending) {
  s->v = view_of(s->tree);
  DeviceScope guard(s->v.device);
  // admit, first come first served
  const int n_old = s->n_act;
  while (!s->queue.empty() && !s->free_bids.empty()) {
    Batch* b = s->queue.front();
    const int64_t s0 = s->slots.take(b->m);
    if (s0 < 0) break;
    s->queue.pop_front();
    const int bid = s->free_bids.back();
    s->free_bids.pop_back();
    b->s0 = s0;
    b->bid = bid;
    bool ok = false;
    const int rc = s->admit(b, s0, bid, &ok);
    if (rc != BKD_OK) {
      s->finish(b, rc);
      return rc;
    }
    if (!ok) {
      s->finish(b, BKD_EINVAL);
      continue;
    }
    b->status = BKD_BATCH_RUNNING;
    b->born = s->rounds;
    s->running[bid] = b;
    s->n_act += (int)b->m;
  }
  if (s->n_act > n_old) {
    const int rc = s->first_round(n_old);
    if (rc != BKD_OK) return rc;
  }
  if (s->n_act > 0) {
    int rc = s->rescue();
    if (rc != BKD_OK) return rc;
    if (s->n_act > 0) {
      rc = s->round();
    } else {
      // every active query was rescued: their batches' counts
      SV_CU(cudaMemcpyAsync(s->h_left, s->batch_left,
                            sizeof(int32_t) * kMaxBatches,
                            cudaMemcpyDeviceToHost, s->v.stream));
      SV_CU(cudaStreamSynchronize(s->v.stream));
    }
    if (rc != BKD_OK) return rc;
    for (int bid = 0; bid < kMaxBatches; ++bid) {
      Batch* b = s->running[bid];
      if (b && s->h_left[bid] == 0) {
        const int rc2 = s->complete(b);
        if (rc2 != BKD_OK) {
          s->finish(b, rc2);
          return rc2;
        }
      }
    }
  }
  if (pending) {
    int64_t n = (int64_t)s->queue.size();
    for (Batch* b : s->running) n += b != nullptr;
    *pending = n;
  }
  return BKD_OK;
}

int cs_status(ClassServer* s, int64_t ticket, int* status) {
  auto it = s->batches.find(ticket);
  if (it == s->batches.end())
    return set_error(BKD_EINVAL, "unknown ticket %lld", (long long)ticket);
  *status = it->second->status;
  if (*status != BKD_BATCH_QUEUED && *status != BKD_BATCH_RUNNING)
    s->batches.erase(it);
  return BKD_OK;
}

}  // namespace

// The public server: one class server per list capacity (k + 1 <= 12, 32,
// 64, up to k_max + 1), each batch routed to the smallest class its k fits,
// so that a k = 1 batch does not carry (and scan with) a k_max + 1 list.
// A ticket is the class server's ticket times kClasses plus the class.
constexpr int kClasses = 3;
constexpr int kClassCap[kClasses] = {12, 32, 64};

struct bkd_server {
  std::vector<std::unique_ptr<ClassServer>> cls;
  std::vector<int> kmax;  // largest k of each class
  int device = 0;
};

extern "C" {

int bkd_serve_open(bkd_tree* t, int k_max, int64_t max_queries,
                   bkd_server** out) {
  set_error(BKD_OK, "");
  if (!out) return set_error(BKD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!t) return set_error(BKD_EINVAL, "tree is NULL");
  if (k_max < 1)
    return set_error(BKD_EINVAL, "k_max must be in [1, n] (got %d)", k_max);
  if (k_max > BKD_MAX_K)
    return set_error(BKD_EUNSUPPORTED, "k_max = %d exceeds BKD_MAX_K = %d",
                     k_max, BKD_MAX_K);
  auto sv = std::make_unique<bkd_server>();
  sv->device = view_of(t).device;
  int lo = 0;
  for (int c = 0; c < kClasses && lo < k_max; ++c) {
    const int kc = std::min(kClassCap[c] - 1, k_max);
    ClassServer* cs = nullptr;
    const int rc = cs_open(t, kc, max_queries, &cs);
    if (rc != BKD_OK) {
      delete cs;
      return rc;
    }
    sv->cls.emplace_back(cs);
    sv->kmax.push_back(kc);
    lo = kc;
  }
  *out = sv.release();
  return BKD_OK;
}

int bkd_serve_submit(bkd_server* s, const float* Q, int64_t m, int k,
                     int64_t* out_idx, float* out_dist, int64_t* ticket) {
  set_error(BKD_OK, "");
  if (!s || !ticket) return set_error(BKD_EINVAL, "server / ticket is NULL");
  const int kmax = s->kmax.empty() ? 0 : s->kmax.back();
  if (k < 1 || k > kmax)
    return set_error(BKD_EINVAL, "k = %d outside [1, k_max = %d]", k, kmax);
  int c = 0;
  while (k > s->kmax[c]) ++c;
  int64_t inner = 0;
  const int rc = cs_submit(s->cls[c].get(), Q, m, k, out_idx, out_dist,
                           &inner);
  if (rc != BKD_OK) return rc;
  *ticket = inner * kClasses + c;
  return BKD_OK;
}

int bkd_serve_step(bkd_server* s, int64_t* pending) {
  set_error(BKD_OK, "");
  if (!s) return set_error(BKD_EINVAL, "server is NULL");
  int64_t total = 0;
  for (auto& cs : s->cls) {
    int64_t p = 0;
    const int rc = cs_step(cs.get(), &p);
    if (rc != BKD_OK) return rc;
    total += p;
  }
  if (pending) *pending = total;
  return BKD_OK;
}

int bkd_serve_status(bkd_server* s, int64_t ticket, int* status) {
  set_error(BKD_OK, "");
  if (!s || !status) return set_error(BKD_EINVAL, "server / status is NULL");
  const int64_t c = ticket % kClasses;
  if (ticket < kClasses || c >= (int64_t)s->cls.size())
    return set_error(BKD_EINVAL, "unknown ticket %lld", (long long)ticket);
  return cs_status(s->cls[c].get(), ticket / kClasses, status);
}

void bkd_serve_close(bkd_server* s) {
  if (!s) return;
  DeviceScope guard(s->device);
  for (auto& cs : s->cls) cudaStreamSynchronize(cs->v.stream);
  delete s;
}

}  // extern "C"
