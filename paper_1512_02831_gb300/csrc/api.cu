// api.cu -- C ABI, device memory, and the LazySearch driver (Algorithm 1).
//
// Query phase, per call (Sec. 2.4, Algorithm 1; Sec. 3.2):
//   init      queries copied and padded, candidate lists +inf, every query
//             in the active list (the `input` queue)
//   round     FindLeafBatch over all active queries -> next leaf or -1;
//             buffer insertion = counting sort of the active queries by
//             leaf id (queries with -1 retire); ProcessAllBuffers over every
//             non-empty buffer; the processed queries form the next round's
//             active list (the `reinsert` queue).  All active queries are
//             fetched every round (M = all, buffers unbounded), so each round
//             triggers ProcessAllBuffers.
//   finish    re-check against the binary64 error bound, binary64 fallback
//             search where needed, results to the caller.
// Chunked ("bigger") mode keeps the leaf structure in pinned host memory and
// runs ProcessAllBuffers chunk by chunk: Brute on the compute stream over
// chunk j while the copy stream moves chunk j+1 into the other device chunk
// buffer, with events in place of the paper's blocking Wait (Sec. 3.2,
// "Brute / Copy / Wait" on two command queues).  Chunks are whole leaves; the
// order alternates direction every round so the chunk processed last stays
// resident for the next round (the paper's prefetch of the first chunk).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "bkd.h"
#include "bkd_internal.h"
#include "chunk_schedule.h"

using namespace bkd;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CU(call)                                                            \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess)                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? BKD_ENOMEM : BKD_ECUDA, \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                  __FILE__, __LINE__);                                      \
  } while (0)

// Where a caller's pointer lives: host memory (pageable or pinned), device
// memory the tree's GPU can use (its own, or managed), or device memory of
// another GPU (rejected: the kernels would read it without peer access).
enum PtrKind { kHostPtr = 0, kDevicePtr = 1, kForeignPtr = -1 };

PtrKind ptr_kind(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return kHostPtr;
  }
  if (a.type == cudaMemoryTypeManaged) return kDevicePtr;
  if (a.type == cudaMemoryTypeDevice)
    return a.device == device ? kDevicePtr : kForeignPtr;
  return kHostPtr;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
      cudaSetDevice(prev);
  }
};

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t count) {
    if (count <= n && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    cudaError_t e = dev_malloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) n = count;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

}  // namespace

struct bkd_tree {
  int device = 0;
  int sm_count = 0;
  cudaStream_t own_stream = nullptr, stream = nullptr, copy_stream = nullptr;
  HostTree host;
  DevTree dev{};
  int64_t n_leaves = 0;
  // resident storage
  float* d_pts = nullptr;
  int64_t* d_orig = nullptr;
  float* d_split = nullptr;
  int32_t* d_leaf_cnt = nullptr;
  float* d_box = nullptr;
  // BF16 screen data (built on request, resident trees only)
  uint16_t* d_scr_words = nullptr;   // tcgen05 screen layout
  uint32_t* d_scr_wwords = nullptr;  // warp screen layout
  float *d_scr_center = nullptr, *d_scr_bmax = nullptr,
        *d_scr_pnmax = nullptr;
  ScreenData screen;
  int precision = 0;
  // chunked storage
  bool chunked = false;
  int n_chunks = 0;
  float* h_pts = nullptr;        // pinned, mapped
  int64_t* h_orig = nullptr;     // pinned, mapped
  std::vector<int32_t> chunk_leaf;   // leaf-aligned chunks: leaf bounds
  bool point_chunks = false;         // chunks split at point positions
  std::vector<int64_t> chunk_pos;    // point chunks: position bounds
  std::vector<int32_t> chunk_la, chunk_lb;  // point chunks: first / last leaf
  int chunk_idx = 0;                 // entries of d_chunk_leaf
  int64_t* d_leaf_lo = nullptr;      // point chunks: leaf bounds (device)
  int32_t* d_chunk_leaf = nullptr;
  float* d_chunk_buf[2] = {nullptr, nullptr};
  int buf_chunk[2] = {-1, -1};
  // chunked trees with the BF16 screen (leaf chunks, warp kernel): the
  // warp layout in pinned host memory, and a device buffer per chunk buffer
  bool chunk_screen = false;
  bool buf_scr[2] = {false, false};  // buffer b holds its chunk's operands
  uint32_t* h_scr_wwords = nullptr;
  uint32_t* d_chunk_scr[2] = {nullptr, nullptr};
  size_t scr_leaf_words = 0;  // words of one leaf in the warp layout
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  // query workspace
  DevBuf<float> qdev, qpad, lst_d;
  DevBuf<uint32_t> lst_i, act_a, act_b, fb_list;
  DevBuf<uint64_t> state;  // per query: TravState
  DevBuf<int2> placed;  // per active position: (next leaf, rank in its buffer)
  DevBuf<int32_t> cnt, off, cursor, toff, chunk_item, nact;
  DevBuf<Item> items, scr_ovf;
  DevBuf<uint8_t> scr_bop;  // screened rounds: per item query operand tile
  DevBuf<uint32_t> scr_seg; // per item survivor segment
  DevBuf<int32_t> scr_cnt;  // per item survivor count
  DevBuf<int64_t> out_idx, inv;
  DevBuf<float> out_dist, score;
  Counters* d_ctr = nullptr;
  Counters* h_ctr = nullptr;     // pinned
  int32_t* h_chunk_item = nullptr;
  uint8_t* d_chunk_done = nullptr;  // per chunk: scanned in the last round
  uint8_t* h_chunk_done = nullptr;  // pinned staging of it
  int max_active = 0;
  int tail_queries = -1;
  int screen_tile = kScreenTile;  // queries per screened work item
  int round_batch = 0;            // rounds per host look (0: automatic)
  int screen_ctas = 0;            // screen CTAs per SM (0: automatic)
  int rescue_rounds = 384;        // server: rounds before the tail rescue
  int defer_queries = 0;          // server: buffer trigger (0: off)
  // timing
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> leaf_ev, copy_ev, tail_ev,
      screen_ev, find_ev, bucket_ev, exact_ev;
  // stats of the last query
  double st_rounds = 0, st_visits = 0, st_pairs = 0, st_resorted = 0,
         st_fallback = 0, st_leaf_ms = 0, st_chunk_bytes = 0, st_copy_ms = 0,
         st_leaf_launches = 0, st_launches = 0, st_tail_queries = 0,
         st_tail_visits = 0, st_tail_pairs = 0, st_tail_ms = 0,
         st_screen_kept = 0, st_screen_pairs = 0, st_screen_ms = 0,
         st_screen_items = 0, st_screen_visits = 0, st_find_ms = 0,
         st_bucket_ms = 0, st_exact_ms = 0, st_chunk_visits = 0,
         st_screen_bytes = 0, st_screen_queued = 0, st_screen_overflow = 0,
         st_leaf_bytes = 0, st_host_syncs = 0, st_fallback_points = 0,
         st_mapped_bytes = 0;

  cudaEvent_t next_event() {
    if (ev_used == ev_pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      ev_pool.push_back(e);
    }
    return ev_pool[ev_used++];
  }
};

namespace {

void release(bkd_tree* t) {
  if (!t) return;
  cudaSetDevice(t->device);
  if (t->stream) cudaStreamSynchronize(t->stream);
  if (t->copy_stream) cudaStreamSynchronize(t->copy_stream);
  cudaFree(t->d_pts);
  cudaFree(t->d_orig);
  cudaFree(t->d_split);
  cudaFree(t->d_leaf_cnt);
  cudaFree(t->d_box);
  cudaFree(t->d_scr_words);
  cudaFree(t->d_scr_wwords);
  cudaFree(t->d_scr_center);
  cudaFree(t->d_scr_bmax);
  cudaFree(t->d_scr_pnmax);
  cudaFree(t->d_chunk_leaf);
  cudaFree(t->d_leaf_lo);
  cudaFree(t->d_chunk_buf[0]);
  cudaFree(t->d_chunk_buf[1]);
  cudaFree(t->d_chunk_scr[0]);
  cudaFree(t->d_chunk_scr[1]);
  if (t->h_scr_wwords) cudaFreeHost(t->h_scr_wwords);
  if (t->h_pts) cudaFreeHost(t->h_pts);
  if (t->h_orig) cudaFreeHost(t->h_orig);
  t->qdev.release();
  t->qpad.release();
  t->lst_d.release();
  t->lst_i.release();
  t->act_a.release();
  t->act_b.release();
  t->fb_list.release();
  t->state.release();
  t->placed.release();
  t->cnt.release();
  t->off.release();
  t->cursor.release();
  t->toff.release();
  t->chunk_item.release();
  t->nact.release();
  t->items.release();
  t->scr_ovf.release();
  t->scr_bop.release();
  t->scr_seg.release();
  t->scr_cnt.release();
  t->out_idx.release();
  t->out_dist.release();
  t->inv.release();
  t->score.release();
  cudaFree(t->d_ctr);
  if (t->h_ctr) cudaFreeHost(t->h_ctr);
  if (t->h_chunk_item) cudaFreeHost(t->h_chunk_item);
  cudaFree(t->d_chunk_done);
  if (t->h_chunk_done) cudaFreeHost(t->h_chunk_done);
  for (auto e : t->ev_pool) cudaEventDestroy(e);
  for (int b = 0; b < 2; ++b) {
    if (t->ev_copied[b]) cudaEventDestroy(t->ev_copied[b]);
    if (t->ev_free[b]) cudaEventDestroy(t->ev_free[b]);
  }
  if (t->own_stream) cudaStreamDestroy(t->own_stream);
  if (t->copy_stream) cudaStreamDestroy(t->copy_stream);
  delete[] t->host.split;
  delete[] t->host.leaf_lo;
  delete[] t->host.perm;
  delete t;
}

// Parallel finiteness / magnitude check of host data.
bool host_values_ok(const float* P, int64_t count) {
  unsigned w = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (count < (1 << 20)) w = 1;
  std::vector<char> ok(w, 1);
  std::vector<std::thread> th;
  for (unsigned i = 0; i < w; ++i)
    th.emplace_back([&, i] {
      const int64_t lo = count * i / w, hi = count * (i + 1) / w;
      for (int64_t j = lo; j < hi; ++j)
        if (!(std::fabs(P[j]) < 1.152921504606846976e18f)) {
          ok[i] = 0;
          break;
        }
    });
  for (auto& x : th) x.join();
  for (char c : ok)
    if (!c) return false;
  return true;
}

int build_impl(const float* P, int64_t n, int d, int height,
               const int64_t* options, int n_options, bkd_tree** out) {
  if (!out) return fail(BKD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!P) return fail(BKD_EINVAL, "P is NULL");
  if (n < 1) return fail(BKD_EINVAL, "n must be >= 1 (got %lld)", (long long)n);
  if (d < 1 || d > BKD_MAX_DIM)
    return fail(BKD_EINVAL, "d must be in [1, %d] (got %d)", BKD_MAX_DIM, d);
  if (height < 0 || height > BKD_MAX_HEIGHT)
    return fail(BKD_EINVAL, "height must be in [0, %d] (got %d)",
                BKD_MAX_HEIGHT, height);
  if (((int64_t)1 << height) > n)
    return fail(BKD_EINVAL, "2^height = %lld leaves exceed n = %lld",
                (long long)((int64_t)1 << height), (long long)n);
  if (n_options < 0 || (n_options > 0 && !options))
    return fail(BKD_EINVAL, "bad options array");
  int64_t cap = -1, chunks = 0, precision = 0, point_chunks = 0,
          screen_kernel = 0;
  for (int i = 0; i < n_options; ++i) {
    const int64_t key = options[2 * i], val = options[2 * i + 1];
    if (key == BKD_OPT_DEVICE_MEM_CAP) {
      if (val < 0) return fail(BKD_EINVAL, "device memory cap must be >= 0");
      cap = val;
    } else if (key == BKD_OPT_CHUNKS) {
      if (val < 0 || val > (1 << 20))
        return fail(BKD_EINVAL, "chunk count out of range");
      chunks = val;
    } else if (key == BKD_OPT_PRECISION) {
      if (val != 0 && val != 1)
        return fail(BKD_EINVAL, "precision must be 0 or 1");
      precision = val;
    } else if (key == BKD_OPT_SCREEN_KERNEL) {
      if (val < 0 || val > 2)
        return fail(BKD_EINVAL, "screen kernel must be 0, 1 or 2");
      screen_kernel = val;
    } else if (key == BKD_OPT_POINT_CHUNKS) {
      if (val != 0 && val != 1)
        return fail(BKD_EINVAL, "point chunks must be 0 or 1");
      point_chunks = val;
    } else if (key == BKD_OPT_STREAM || key == BKD_OPT_MAX_ACTIVE ||
               key == BKD_OPT_TAIL_QUERIES || key == BKD_OPT_SCREEN_TILE ||
               key == BKD_OPT_ROUND_BATCH || key == BKD_OPT_SCREEN_CTAS ||
               key == BKD_OPT_RESCUE_ROUNDS || key == BKD_OPT_DEFER_QUERIES) {
      // applied after construction below
    } else {
      return fail(BKD_EINVAL, "unknown build option %lld", (long long)key);
    }
  }

  bkd_tree* t = new (std::nothrow) bkd_tree();
  if (!t) return fail(BKD_ENOMEM, "host allocation failed");
  auto bail = [&](int code) {
    release(t);
    return code;
  };
  if (cudaGetDevice(&t->device) != cudaSuccess)
    return bail(fail(BKD_ECUDA, "no CUDA device"));
  cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount,
                         t->device);
  if (cudaStreamCreateWithFlags(&t->own_stream, cudaStreamNonBlocking) !=
          cudaSuccess ||
      cudaStreamCreateWithFlags(&t->copy_stream, cudaStreamNonBlocking) !=
          cudaSuccess)
    return bail(fail(BKD_ECUDA, "stream creation failed"));
  t->stream = t->own_stream;

  // points on the host
  std::vector<float> hostP;
  const float* Ph = P;
  const PtrKind pk = ptr_kind(P, t->device);
  if (pk == kForeignPtr)
    return bail(fail(BKD_EINVAL, "P is device memory of another GPU than "
                                 "the current device %d", t->device));
  if (pk == kDevicePtr) {
    try {
      hostP.resize((size_t)(n * d));
    } catch (...) {
      return bail(fail(BKD_ENOMEM, "host copy of P failed"));
    }
    if (cudaMemcpy(hostP.data(), P, sizeof(float) * n * d,
                   cudaMemcpyDeviceToHost) != cudaSuccess)
      return bail(fail(BKD_ECUDA, "copy of P to the host failed"));
    Ph = hostP.data();
  }
  if (!host_values_ok(Ph, n * d))
    return bail(fail(BKD_EINVAL, "P holds a non-finite or |x| >= 2^60 value"));

  if (const char* msg = build_host_tree(Ph, n, d, height, &t->host))
    return bail(fail(BKD_ENOMEM, "%s", msg));
  HostTree& H = t->host;
  const int64_t L = (int64_t)1 << height;
  t->n_leaves = L;
  const int64_t slots = L * H.lcap;
  if (slots >= (int64_t)0xffffffff)
    return bail(fail(BKD_EUNSUPPORTED,
                     "leaf structure of %lld slots exceeds 2^32 - 1",
                     (long long)slots));
  const size_t pts_bytes = (size_t)slots * H.Dp * sizeof(float);
  const size_t orig_bytes = (size_t)slots * sizeof(int64_t);

  // choose resident or chunked mode
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  if (cap < 0) cap = (int64_t)(0.6 * (double)free_b);
  bool chunked = chunks >= 1 || (int64_t)pts_bytes > cap;
  if (chunked && chunks == 0) {
    for (chunks = 2; chunks < L; ++chunks) {
      const int64_t leaves = (L + chunks - 1) / chunks;
      if (2 * leaves * H.lcap * H.Dp * 4 <= cap) break;
    }
    chunks = std::min<int64_t>(chunks, L);
  }
  if (chunked) chunks = std::min<int64_t>(chunks, L);
  t->chunked = chunked;
  t->n_chunks = chunked ? (int)chunks : 0;

  // split values and leaf sizes
  std::vector<int32_t> leaf_cnt(L);
  for (int64_t l = 0; l < L; ++l)
    leaf_cnt[l] = (int32_t)(H.leaf_lo[l + 1] - H.leaf_lo[l]);
  const int64_t nsplit = std::max<int64_t>(L - 1, 1);
  if (dev_malloc(&t->d_split, nsplit * sizeof(float)) != cudaSuccess ||
      dev_malloc(&t->d_leaf_cnt, L * sizeof(int32_t)) != cudaSuccess)
    return bail(fail(BKD_ENOMEM, "device allocation failed (tree)"));
  {
    const int64_t nodes = 2 * L - 1;
    std::vector<float> box;
    try {
      box.resize((size_t)nodes * 2 * H.Dp);
    } catch (...) {
      return bail(fail(BKD_ENOMEM, "host allocation failed (boxes)"));
    }
    fill_boxes(Ph, H, box.data());
    if (dev_malloc(&t->d_box, box.size() * sizeof(float)) != cudaSuccess)
      return bail(fail(BKD_ENOMEM, "device allocation failed (boxes)"));
    if (cudaMemcpy(t->d_box, box.data(), box.size() * sizeof(float),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(BKD_ECUDA, "upload of the node boxes failed"));
  }
  if (cudaMemcpy(t->d_split, H.split, nsplit * sizeof(float),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(t->d_leaf_cnt, leaf_cnt.data(), L * sizeof(int32_t),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(BKD_ECUDA, "upload of the top tree failed"));

  if (!chunked) {
    std::vector<float> qbuf;
    std::vector<int64_t> obuf;
    try {
      qbuf.resize(pts_bytes / sizeof(float));
      obuf.resize(slots);
    } catch (...) {
      return bail(fail(BKD_ENOMEM, "host staging of the leaf structure"));
    }
    fill_quads(Ph, H, 0, L, qbuf.data(), obuf.data());
    if (dev_malloc(&t->d_pts, pts_bytes) != cudaSuccess ||
        dev_malloc(&t->d_orig, orig_bytes) != cudaSuccess)
      return bail(fail(BKD_ENOMEM, "device allocation of %zu bytes failed",
                       pts_bytes + orig_bytes));
    if (cudaMemcpy(t->d_pts, qbuf.data(), pts_bytes, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(t->d_orig, obuf.data(), orig_bytes,
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(BKD_ECUDA, "upload of the leaf structure failed"));
  } else {
    if (host_alloc(&t->h_pts, pts_bytes,
                      cudaHostAllocMapped | cudaHostAllocPortable) !=
            cudaSuccess ||
        host_alloc(&t->h_orig, orig_bytes,
                      cudaHostAllocMapped | cudaHostAllocPortable) !=
            cudaSuccess) {
      cudaGetLastError();
      return bail(fail(BKD_ENOMEM, "pinned host allocation of %zu bytes failed",
                       pts_bytes + orig_bytes));
    }
    fill_quads(Ph, H, 0, L, t->h_pts, t->h_orig);
    const int N = t->n_chunks;
    int64_t max_leaves = 0;
    std::vector<int32_t> idx;  // leaves whose first item / query bound a
                               // chunk's items and queries
    if (!point_chunks) {
      t->chunk_leaf.resize(N + 1);
      for (int c = 0; c <= N; ++c)  // C_c = ceil(c L / N), leaves
        t->chunk_leaf[c] = (int32_t)((c * L + N - 1) / N);
      for (int c = 0; c < N; ++c)
        max_leaves = std::max<int64_t>(max_leaves,
                                       t->chunk_leaf[c + 1] - t->chunk_leaf[c]);
      idx = t->chunk_leaf;
    } else {
      // Sec. 3.2: C_j holds the leaf-structure positions [ceil(j n / N),
      // ceil((j + 1) n / N)); a bound inside a leaf moves down to the start
      // of its group of four points (the quads the leaf kernel reads), so
      // every chunk takes whole quads and every point lies in one chunk
      auto leaf_of = [&](int64_t p) {
        return (int32_t)(std::upper_bound(H.leaf_lo, H.leaf_lo + L + 1, p) -
                         H.leaf_lo - 1);
      };
      t->chunk_pos.resize(N + 1);
      for (int j = 0; j <= N; ++j) {
        const int64_t p = (j * n + N - 1) / N;
        if (j == 0 || j == N) {
          t->chunk_pos[j] = p;
          continue;
        }
        const int64_t b = H.leaf_lo[leaf_of(p)];
        t->chunk_pos[j] = b + ((p - b) & ~(int64_t)3);
      }
      for (int j = 0; j < N; ++j)
        if (t->chunk_pos[j + 1] <= t->chunk_pos[j])
          return bail(fail(BKD_EINVAL, "%d point chunks are too many for n = "
                                       "%lld points", N, (long long)n));
      t->chunk_la.resize(N);
      t->chunk_lb.resize(N);
      for (int j = 0; j < N; ++j) {
        t->chunk_la[j] = leaf_of(t->chunk_pos[j]);
        t->chunk_lb[j] = leaf_of(t->chunk_pos[j + 1] - 1);
        max_leaves = std::max<int64_t>(max_leaves,
                                       t->chunk_lb[j] - t->chunk_la[j] + 1);
        idx.push_back(t->chunk_la[j]);
        idx.push_back(t->chunk_lb[j] + 1);
      }
      if (dev_malloc(&t->d_leaf_lo, (L + 1) * sizeof(int64_t)) != cudaSuccess)
        return bail(fail(BKD_ENOMEM, "device leaf bounds"));
      if (cudaMemcpy(t->d_leaf_lo, H.leaf_lo, (L + 1) * sizeof(int64_t),
                     cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(BKD_ECUDA, "upload of leaf bounds failed"));
    }
    t->point_chunks = point_chunks != 0;
    t->chunk_idx = (int)idx.size();
    const size_t buf_bytes = (size_t)max_leaves * H.lcap * H.Dp * sizeof(float);
    if (dev_malloc(&t->d_chunk_buf[0], buf_bytes) != cudaSuccess ||
        dev_malloc(&t->d_chunk_buf[1], buf_bytes) != cudaSuccess ||
        dev_malloc(&t->d_chunk_leaf, idx.size() * sizeof(int32_t)) !=
            cudaSuccess)
      return bail(fail(BKD_ENOMEM, "device chunk buffers (%zu bytes each)",
                       buf_bytes));
    if (cudaMemcpy(t->d_chunk_leaf, idx.data(), idx.size() * sizeof(int32_t),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(BKD_ECUDA, "upload of chunk bounds failed"));
    for (int b = 0; b < 2; ++b)
      if (cudaEventCreateWithFlags(&t->ev_copied[b], cudaEventDisableTiming) !=
              cudaSuccess ||
          cudaEventCreateWithFlags(&t->ev_free[b], cudaEventDisableTiming) !=
              cudaSuccess)
        return bail(fail(BKD_ECUDA, "event creation failed"));
  }
  if (precision == 1) {
    // chunked trees: leaf chunks and the warp kernel only (its point layout
    // is streamed with the points, chunk by chunk)
    if (chunked && (point_chunks || screen_kernel == 1))
      return bail(fail(BKD_EUNSUPPORTED,
                       "the BF16 screen on a chunked tree needs leaf chunks "
                       "(BKD_OPT_POINT_CHUNKS=0) and the warp screen kernel "
                       "(BKD_OPT_SCREEN_KERNEL=0)"));
    if (chunked) screen_kernel = 0;
    // the layouts of the screen kernels asked for: 0 the warp kernel, 1
    // the tcgen05 kernel, 2 both (the warp kernel runs; BKD_OPT_SCREEN_KERNEL
    // switches)
    const bool want_warp = screen_kernel != 1, want_tc = screen_kernel != 0;
    const int kh = screen_halves(d), wkh = screen_halves_warp(d);
    const int64_t tiles = screen_tiles(H.lcap);
    const int64_t stride = screen_stride(H.lcap);
    std::vector<uint16_t> words;
    std::vector<uint32_t> wwords;
    std::vector<float> center, bmax, pnmax;
    try {
      if (want_tc) words.resize((size_t)L * tiles * kScreenRows * 16 * kh);
      if (want_warp && !chunked) wwords.resize((size_t)L * wkh * stride * 8);
      center.resize((size_t)L * d);
      bmax.resize(L);
      pnmax.resize(L);
    } catch (...) {
      return bail(fail(BKD_ENOMEM, "host staging of the screen data"));
    }
    if (want_tc)
      fill_screen(Ph, H, tiles, words.data(), center.data(), bmax.data(),
                  pnmax.data());
    t->scr_leaf_words = (size_t)wkh * stride * 8;
    if (want_warp && chunked) {
      // pinned host copy streamed with the chunks; a device buffer per chunk
      // buffer, as large as the largest chunk
      const size_t hb = (size_t)L * t->scr_leaf_words * 4;
      int64_t max_leaves = 0;
      for (int c = 0; c < t->n_chunks; ++c)
        max_leaves = std::max<int64_t>(max_leaves, t->chunk_leaf[c + 1] -
                                                       t->chunk_leaf[c]);
      const size_t db = (size_t)max_leaves * t->scr_leaf_words * 4;
      if (host_alloc(&t->h_scr_wwords, hb, cudaHostAllocPortable) !=
              cudaSuccess ||
          dev_malloc(&t->d_chunk_scr[0], db) != cudaSuccess ||
          dev_malloc(&t->d_chunk_scr[1], db) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(BKD_ENOMEM, "screen chunk buffers"));
      }
      fill_screen_warp(Ph, H, stride, t->h_scr_wwords, center.data(),
                       bmax.data(), pnmax.data());
      t->chunk_screen = true;
    } else if (want_warp) {
      fill_screen_warp(Ph, H, stride, wwords.data(), center.data(),
                       bmax.data(), pnmax.data());
    }
    if ((want_tc &&
         dev_malloc(&t->d_scr_words, words.size() * 2) != cudaSuccess) ||
        (want_warp && !chunked &&
         dev_malloc(&t->d_scr_wwords, wwords.size() * 4) != cudaSuccess) ||
        dev_malloc(&t->d_scr_center, center.size() * 4) != cudaSuccess ||
        dev_malloc(&t->d_scr_bmax, bmax.size() * 4) != cudaSuccess ||
        dev_malloc(&t->d_scr_pnmax, pnmax.size() * 4) != cudaSuccess)
      return bail(fail(BKD_ENOMEM, "device allocation failed (screen data)"));
    if ((want_tc &&
         cudaMemcpy(t->d_scr_words, words.data(), words.size() * 2,
                    cudaMemcpyHostToDevice) != cudaSuccess) ||
        (want_warp && !chunked &&
         cudaMemcpy(t->d_scr_wwords, wwords.data(), wwords.size() * 4,
                    cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy(t->d_scr_center, center.data(), center.size() * 4,
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->d_scr_bmax, bmax.data(), bmax.size() * 4,
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->d_scr_pnmax, pnmax.data(), pnmax.size() * 4,
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(BKD_ECUDA, "upload of the screen data failed"));
    t->screen.words = t->d_scr_words;
    // (chunked: a chunk buffer stands for the layout; every launch passes
    // the buffer of its chunk)
    t->screen.wwords = chunked ? t->d_chunk_scr[0] : t->d_scr_wwords;
    t->screen.tiles = tiles;
    t->screen.stride = stride;
    t->screen.center = t->d_scr_center;
    t->screen.bmax = t->d_scr_bmax;
    t->screen.pnmax = t->d_scr_pnmax;
    t->screen.kh = kh;
    t->screen.wkh = wkh;
    t->screen.kind = want_warp ? 0 : 1;
    t->screen_tile = screen_tile_of(t->screen.kind);
    t->precision = 1;
  }
  if (dev_malloc(&t->d_ctr, sizeof(Counters)) != cudaSuccess ||
      host_alloc(&t->h_ctr, sizeof(Counters), cudaHostAllocDefault) !=
          cudaSuccess ||
      host_alloc(&t->h_chunk_item,
                 2 * (size_t)std::max(t->chunk_idx, 1) * sizeof(int32_t),
                    cudaHostAllocDefault) != cudaSuccess ||
      (chunked &&
       (dev_malloc(&t->d_chunk_done, t->n_chunks) != cudaSuccess ||
        host_alloc(&t->h_chunk_done, t->n_chunks, cudaHostAllocDefault) !=
            cudaSuccess)))
    return bail(fail(BKD_ENOMEM, "counter allocation failed"));

  DevTree& D = t->dev;
  D.split = t->d_split;
  D.pts = chunked ? t->h_pts : t->d_pts;
  D.orig = chunked ? t->h_orig : t->d_orig;
  D.leaf_cnt = t->d_leaf_cnt;
  D.box = t->d_box;
  D.n = n;
  D.d = d;
  D.Dp = H.Dp;
  D.h = height;
  D.lcap = H.lcap;
  D.n_chunks = t->n_chunks;
  D.chunk_done = chunked && !t->point_chunks ? t->d_chunk_done : nullptr;
  for (int i = 0; i < n_options; ++i) {
    const int64_t key = options[2 * i], val = options[2 * i + 1];
    if (key == BKD_OPT_STREAM || key == BKD_OPT_MAX_ACTIVE ||
        key == BKD_OPT_TAIL_QUERIES || key == BKD_OPT_SCREEN_TILE ||
        key == BKD_OPT_ROUND_BATCH || key == BKD_OPT_SCREEN_CTAS ||
        key == BKD_OPT_RESCUE_ROUNDS || key == BKD_OPT_DEFER_QUERIES) {
      int rc = bkd_set_option(t, (int)key, val);
      if (rc != BKD_OK) return bail(rc);
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess)
    return bail(fail(BKD_ECUDA, "build failed: %s",
                     cudaGetErrorString(cudaGetLastError())));
  *out = t;
  return BKD_OK;
}

void reset_stats(bkd_tree* t) {
  t->st_rounds = t->st_visits = t->st_pairs = t->st_resorted =
      t->st_fallback = t->st_leaf_ms = t->st_chunk_bytes = t->st_copy_ms =
          t->st_leaf_launches = t->st_launches = t->st_tail_queries =
              t->st_tail_visits = t->st_tail_pairs = t->st_tail_ms =
                  t->st_screen_kept = t->st_screen_pairs = t->st_screen_ms = 0;
  t->st_screen_items = t->st_screen_visits = 0;
  t->st_find_ms = t->st_bucket_ms = t->st_exact_ms = 0;
  t->st_chunk_visits = t->st_screen_bytes = t->st_leaf_bytes = 0;
  t->st_host_syncs = t->st_fallback_points = t->st_mapped_bytes = 0;
  t->st_screen_queued = t->st_screen_overflow = 0;
  t->ev_used = 0;
  t->find_ev.clear();
  t->bucket_ev.clear();
  t->exact_ev.clear();
  t->leaf_ev.clear();
  t->copy_ev.clear();
  t->tail_ev.clear();
  t->screen_ev.clear();
}

// Sums the CUDA-event timings of the last call into the stats.
void collect_timings(bkd_tree* t) {
  const std::pair<std::vector<std::pair<cudaEvent_t, cudaEvent_t>>*,
                  double*>
      phases[] = {{&t->leaf_ev, &t->st_leaf_ms},
                  {&t->copy_ev, &t->st_copy_ms},
                  {&t->tail_ev, &t->st_tail_ms},
                  {&t->screen_ev, &t->st_screen_ms},
                  {&t->find_ev, &t->st_find_ms},
                  {&t->bucket_ev, &t->st_bucket_ms},
                  {&t->exact_ev, &t->st_exact_ms}};
  for (const auto& ph : phases)
    for (auto& pr : *ph.first) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess)
        *ph.second += ms;
    }
  cudaGetLastError();
}

// One LazySearch over queries already in t->qdev[0..m) (row-major m x d).
// Results go to device buffers out_idx / out_dist.
int search(bkd_tree* t, int64_t m, int k, int64_t* out_idx, float* out_dist) {
  const int K = k + 1;
  const int cap = list_capacity(K);
  const DevTree& D = t->dev;
  const int Dp = D.Dp;
  cudaStream_t s = t->stream;
  const int64_t L = t->n_leaves;
  const int64_t max_items =
      m / std::min(t->screen_tile, kPipeTile) + L + 1;  // items of any round
  CU(t->qpad.ensure(m * Dp));
  CU(t->lst_d.ensure(m * K));
  CU(t->lst_i.ensure(m * K));
  CU(t->state.ensure(m));
  CU(t->act_a.ensure(m));
  CU(t->act_b.ensure(m));
  CU(t->placed.ensure(m));
  CU(t->fb_list.ensure(m));
  CU(t->cnt.ensure(L));
  CU(t->cursor.ensure(std::max<int64_t>(L, 4)));  // also holds the scan's tile sums
  CU(t->off.ensure(L + 1));
  CU(t->toff.ensure(L + 1));
  CU(t->items.ensure(max_items));
  CU(t->nact.ensure(2));
  if (t->chunked) CU(t->chunk_item.ensure(2 * t->chunk_idx));

  CU(cudaMemsetAsync(t->d_ctr, 0, sizeof(Counters), s));
  CU(launch_init(t->qdev.p, m, D.d, Dp, t->qpad.p, t->lst_d.p, t->lst_i.p, K,
                 t->state.p, t->act_a.p, 0u, t->d_ctr, s));
  t->st_launches += 1;
  // reject non-finite queries before any traversal (the tail kernel may take
  // every query without a single round)
  CU(cudaMemcpyAsync(t->h_ctr, t->d_ctr, sizeof(Counters),
                     cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (t->h_ctr->err & kErrNonFinite)
    return fail(BKD_EINVAL, "Q holds a non-finite or |x| >= 2^60 value");
  uint32_t* act = t->act_a.p;
  uint32_t* nxt = t->act_b.p;
  int n_act = (int)m;
  const int grid_max = leaf_kernel_grid(Dp, cap, t->sm_count);
  int screen_max =
      t->precision == 1
          ? screen_grid(t->screen, Dp, D.lcap, K, t->sm_count)
                        : 0;
  if (t->screen_ctas > 0)
    screen_max = std::min(screen_max, t->screen_ctas * t->sm_count);
  // the tail kernel spreads a list over the 32 lanes of a warp (two
  // entries per lane above 32); automatic threshold: 8,192 active queries, up to 32,768 for the largest query
  // sets (measured on 2^24 queries)
  const int64_t tail_auto =
      std::max<int64_t>(8192, std::min<int64_t>(32768, m / 512));
  const int tail =
      (int)(t->tail_queries >= 0 ? t->tail_queries : tail_auto);
  // A round: FindLeafBatch over the active queries (it also counts every
  // query into its next leaf), bucketing by leaf, ProcessAllBuffers.  The
  // host looks at the counters after a round's bucketing (all done: stop;
  // few left: tail kernel).  On a resident tree it then queues a batch of
  // further rounds without waiting: their kernels read the active and item
  // counts on the device, and a round whose queries have all finished does
  // nothing.  A chunked tree needs the host every round (the chunk
  // schedule).
  ScreenWork sw;
  if (screen_max > 0 && t->screen.kind == 1) {
    const int64_t si = m / t->screen_tile + L + 1;  // items of a screened round
    CU(t->scr_bop.ensure(si * 4096 * t->screen.kh));
    CU(t->scr_seg.ensure(si * screen_seg_cap()));
    CU(t->scr_cnt.ensure(si * screen_cnt_per_item()));
    CU(t->scr_ovf.ensure(2 * si));  // overflowed items, in halves
    sw.bop = t->scr_bop.p;
    sw.seg = t->scr_seg.p;
    sw.seg_cnt = t->scr_cnt.p;
    sw.ovf = t->scr_ovf.p;
  }
  int round = 0;
  CU(launch_fill(t->nact.p, 1, (int32_t)m, s));
  t->st_launches += 1;
  auto start_round = [&](bool dev_counts) -> int {
    // a round that ends in the BF16 screen (the first round stays on the
    // float32 kernel: every list is still empty there) buckets its queries
    // into the screen's items
    const bool screened = (!t->chunked || t->chunk_screen) &&
                          t->precision == 1 && round > 0 && screen_max > 0;
    const int32_t* nin = dev_counts ? t->nact.p + (round & 1) : nullptr;
    int32_t* nout = t->nact.p + ((round + 1) & 1);
    cudaEvent_t f0 = t->next_event(), f1 = t->next_event();
    if (f0) cudaEventRecord(f0, s);
    CU(cudaMemsetAsync(t->cnt.p, 0, sizeof(int32_t) * L, s));
    CU(launch_find_leaf(D, t->qpad.p, act, n_act, t->state.p, t->lst_d.p, K,
                        t->placed.p, t->cnt.p, s, nin));
    if (f1) cudaEventRecord(f1, s);
    if (f0 && f1) t->find_ev.push_back({f0, f1});
    t->st_launches += 1;
    cudaEvent_t b0 = t->next_event(), b1 = t->next_event();
    if (b0) cudaEventRecord(b0, s);
    CU(launch_bucket(t->placed.p, act, n_act, (int)L,
                     screened ? t->screen_tile : kPipeTile,
                     t->d_leaf_cnt, t->cnt.p, t->off.p, t->cursor.p,
                     t->toff.p, t->items.p, nxt, t->d_ctr, s, nin, nout));
    if (b1) cudaEventRecord(b1, s);
    if (b0 && b1) t->bucket_ev.push_back({b0, b1});
    t->st_launches += 3;
    if (t->chunked) {
      CU(launch_chunk_items(t->toff.p, t->off.p, t->d_chunk_leaf,
                            t->chunk_idx, t->chunk_item.p, s));
      CU(cudaMemcpyAsync(t->h_chunk_item, t->chunk_item.p,
                         2 * t->chunk_idx * sizeof(int32_t),
                         cudaMemcpyDeviceToHost, s));
      t->st_launches += 1;
    }
    return BKD_OK;
  };
  // ProcessAllBuffers of the round just bucketed (n_items < 0: the count is
  // read on the device), then the bucketed list becomes the active list
  auto process_round = [&](int n_items) -> int {
    const bool screened = (!t->chunked || t->chunk_screen) &&
                          t->precision == 1 && round > 0 && screen_max > 0;
    if (screened && !t->chunked) {
      // BF16 tensor-core screen + exact float32 rescoring
      cudaEvent_t e0 = t->next_event(), e1 = t->next_event();
      if (e0) cudaEventRecord(e0, s);
      CU(launch_screen(D, t->screen, t->items.p, n_items, t->d_ctr, nxt,
                       t->qpad.p, t->lst_d.p, t->lst_i.p, K, screen_max, sw,
                       cap, grid_max, t->sm_count, s));
      if (e1) cudaEventRecord(e1, s);
      if (e0 && e1) t->screen_ev.push_back({e0, e1});
      t->st_launches += 1;
    } else if (!t->chunked) {
      const int grid = n_items >= 0 ? std::min(grid_max, n_items) : grid_max;
      cudaEvent_t e0 = t->next_event(), e1 = t->next_event();
      if (e0) cudaEventRecord(e0, s);
      CU(launch_leaf(D, cap, t->items.p, 0, n_items, t->d_ctr, t->d_pts, 0,
                     nxt, t->qpad.p, t->lst_d.p, t->lst_i.p, K, grid, s));
      if (e1) cudaEventRecord(e1, s);
      if (e0 && e1) t->leaf_ev.push_back({e0, e1});
      t->st_leaf_launches += 1;
      t->st_launches += 1;
    } else if (t->point_chunks) {
      // Brute / Copy / Wait (Sec. 3.2) with the paper's point chunks: every
      // chunk whose leaves hold buffered queries, in order (alternating
      // direction, so the chunk scanned last stays resident); a query whose
      // leaf straddles two chunks is scanned in both, each time against the
      // leaf's points inside the chunk.
      const int N = t->n_chunks;
      const int32_t* ci = t->h_chunk_item;  // [first item, end item) per chunk
      int prev_b = -1;
      for (int i = 0; i < N; ++i) {
        const int c = point_chunk_at(round, i, N);
        const int ilo = ci[2 * c], ihi = ci[2 * c + 1];
        if (ihi <= ilo) continue;
        const int b = point_chunk_buffer(c, t->buf_chunk, prev_b);
        const int64_t la = t->chunk_la[c], lb = t->chunk_lb[c] + 1;
        if (t->buf_chunk[b] != c) {
          const size_t bytes = (size_t)(lb - la) * D.lcap * Dp * sizeof(float);
          CU(cudaStreamWaitEvent(t->copy_stream, t->ev_free[b], 0));
          cudaEvent_t c0 = t->next_event(), c1 = t->next_event();
          if (c0) cudaEventRecord(c0, t->copy_stream);
          CU(cudaMemcpyAsync(t->d_chunk_buf[b],
                             t->h_pts + (size_t)la * D.lcap * Dp, bytes,
                             cudaMemcpyHostToDevice, t->copy_stream));
          if (c1) cudaEventRecord(c1, t->copy_stream);
          if (c0 && c1) t->copy_ev.push_back({c0, c1});
          CU(cudaEventRecord(t->ev_copied[b], t->copy_stream));
          t->buf_chunk[b] = c;
          t->st_chunk_bytes += (double)bytes;
        }
        CU(cudaStreamWaitEvent(s, t->ev_copied[b], 0));
        LeafPart part;
        part.leaf_lo = t->d_leaf_lo;
        part.pos_lo = t->chunk_pos[c];
        part.pos_hi = t->chunk_pos[c + 1];
        cudaEvent_t e0 = t->next_event(), e1 = t->next_event();
        if (e0) cudaEventRecord(e0, s);
        CU(launch_leaf(D, cap, t->items.p, ilo, ihi, t->d_ctr,
                       t->d_chunk_buf[b], la, nxt, t->qpad.p, t->lst_d.p,
                       t->lst_i.p, K, std::min(grid_max, ihi - ilo), s,
                       nullptr, part));
        if (e1) cudaEventRecord(e1, s);
        if (e0 && e1) t->leaf_ev.push_back({e0, e1});
        CU(cudaEventRecord(t->ev_free[b], s));
        t->st_leaf_launches += 1;
        t->st_launches += 1;
        prev_b = b;
      }
    } else {
      // Brute / Copy / Wait (Sec. 3.2) on the chunks the schedule picks.
      // The paper streams every chunk in every ProcessAllBuffers call and
      // relies on its half-full trigger to make calls rare; here a round
      // keeps running the two chunks resident in the device buffers while
      // their buffers hold queries (traversals move mostly between nearby
      // leaves, which share a chunk), and brings in the chunk with the most
      // buffered queries when a buffer is empty or that chunk holds more
      // than twice the resident work.  Queries buffered in other chunks
      // wait there (FindLeafBatch re-places them) until their chunk comes
      // in.  Results do not depend on the schedule.
      const int N = t->n_chunks;
      const int32_t* ci = t->h_chunk_item;          // first item per chunk
      const int32_t* cq = t->h_chunk_item + N + 1;  // first query per chunk
      auto work = [&](int c) { return c < 0 ? 0 : cq[c + 1] - cq[c]; };
      const ChunkLoad pick = pick_leaf_chunk_load(N, t->buf_chunk, work);
      const int load_b = pick.buffer;
      if (load_b >= 0) {
        const int c = pick.chunk;
        const int64_t leaf_a = t->chunk_leaf[c], leaf_b = t->chunk_leaf[c + 1];
        const size_t off_f = (size_t)leaf_a * D.lcap * Dp;
        const size_t bytes =
            (size_t)(leaf_b - leaf_a) * D.lcap * Dp * sizeof(float);
        CU(cudaStreamWaitEvent(t->copy_stream, t->ev_free[load_b], 0));
        cudaEvent_t c0 = t->next_event(), c1 = t->next_event();
        if (c0) cudaEventRecord(c0, t->copy_stream);
        CU(cudaMemcpyAsync(t->d_chunk_buf[load_b], t->h_pts + off_f, bytes,
                           cudaMemcpyHostToDevice, t->copy_stream));
        t->buf_scr[load_b] = false;
        if (t->chunk_screen && t->precision == 1) {
          // the chunk's screen operands travel with its points
          const size_t sb = (size_t)(leaf_b - leaf_a) * t->scr_leaf_words * 4;
          CU(cudaMemcpyAsync(t->d_chunk_scr[load_b],
                             t->h_scr_wwords + (size_t)leaf_a *
                                                   t->scr_leaf_words,
                             sb, cudaMemcpyHostToDevice, t->copy_stream));
          t->st_chunk_bytes += (double)sb;
          t->buf_scr[load_b] = true;
        }
        if (c1) cudaEventRecord(c1, t->copy_stream);
        if (c0 && c1) t->copy_ev.push_back({c0, c1});
        CU(cudaEventRecord(t->ev_copied[load_b], t->copy_stream));
        t->buf_chunk[load_b] = c;
        t->st_chunk_bytes += (double)bytes;
      }
      std::fill(t->h_chunk_done, t->h_chunk_done + N, (uint8_t)0);
      // the retained chunk first: its Brute hides the Copy of the other
      const int order[2] = {load_b == 0 ? 1 : 0, load_b == 0 ? 0 : 1};
      for (int b : order) {
        const int c = t->buf_chunk[b];
        if (c < 0 || work(c) == 0) continue;
        const int ilo = ci[c], ihi = ci[c + 1];
        CU(cudaStreamWaitEvent(s, t->ev_copied[b], 0));
        cudaEvent_t e0 = t->next_event(), e1 = t->next_event();
        if (e0) cudaEventRecord(e0, s);
        if (screened) {
          // the warp screen over the chunk in buffer b: its points and
          // screen operands start at the chunk's first leaf
          DevTree Dc = D;
          Dc.pts = t->d_chunk_buf[b];
          ScreenData sc = t->screen;
          sc.wwords = t->d_chunk_scr[b];
          sc.leaf0 = t->chunk_leaf[c];
          CU(launch_screen_warp(Dc, sc, t->items.p, ilo, ihi, t->d_ctr, nxt,
                                t->qpad.p, t->lst_d.p, t->lst_i.p, K,
                                screen_max, s));
        } else {
          const int grid = std::min(grid_max, ihi - ilo);
          CU(launch_leaf(D, cap, t->items.p, ilo, ihi, t->d_ctr,
                         t->d_chunk_buf[b], t->chunk_leaf[c], nxt, t->qpad.p,
                         t->lst_d.p, t->lst_i.p, K, grid, s));
        }
        if (e1) cudaEventRecord(e1, s);
        if (e0 && e1)
          (screened ? t->screen_ev : t->leaf_ev).push_back({e0, e1});
        CU(cudaEventRecord(t->ev_free[b], s));
        t->h_chunk_done[c] = 1;
        t->st_chunk_visits += work(c);
        if (!screened) t->st_leaf_launches += 1;
        t->st_launches += 1;
      }
      // which chunks this round scanned, for the next FindLeafBatch
      CU(cudaMemcpyAsync(t->d_chunk_done, t->h_chunk_done, N,
                         cudaMemcpyHostToDevice, s));
    }
    t->st_rounds += 1;
    std::swap(act, nxt);
    ++round;
    return BKD_OK;
  };
  // a chunk left resident by a float32 call has no screen operands in its
  // buffer yet: copy them before this call screens it
  if (t->chunk_screen && t->precision == 1 && !t->point_chunks)
    for (int b = 0; b < 2; ++b) {
      const int c = t->buf_chunk[b];
      if (c < 0 || t->buf_scr[b]) continue;
      const int64_t leaf_a = t->chunk_leaf[c], leaf_b = t->chunk_leaf[c + 1];
      const size_t sb = (size_t)(leaf_b - leaf_a) * t->scr_leaf_words * 4;
      CU(cudaStreamWaitEvent(t->copy_stream, t->ev_free[b], 0));
      CU(cudaMemcpyAsync(t->d_chunk_scr[b],
                         t->h_scr_wwords + (size_t)leaf_a * t->scr_leaf_words,
                         sb, cudaMemcpyHostToDevice, t->copy_stream));
      CU(cudaEventRecord(t->ev_copied[b], t->copy_stream));
      t->st_chunk_bytes += (double)sb;
      t->buf_scr[b] = true;
    }
  int rc = start_round(false);
  if (rc != BKD_OK) return rc;
  // bucketing totals of the first round (float32 kernel) and of the last
  // (not processed: everything done, or handed to the tail kernel)
  unsigned long long first_pairs = 0, first_items = 0, first_visits = 0;
  unsigned long long last_pairs = 0, last_items = 0, last_visits = 0;
  for (bool first = true;; first = false) {
    CU(cudaMemcpyAsync(t->h_ctr, t->d_ctr, sizeof(Counters),
                       cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    t->st_host_syncs += 1;
    if (t->h_ctr->err & kErrTimeout)
      return fail(BKD_ETIMEOUT, "a bounded device-side wait ran out");
    const int n_next = t->h_ctr->n_next;
    const int n_items = t->h_ctr->n_items;
    last_pairs = t->h_ctr->pairs;
    last_items = (unsigned long long)n_items;
    last_visits = (unsigned long long)n_next;
    if (first) {
      first_pairs = last_pairs;
      first_items = last_items;
      first_visits = last_visits;
    }
    if (n_next == 0) break;
    if (n_next <= tail) {
      // finish the remaining queries in one launch, one warp per query,
      // starting from each one's pending leaf
      cudaEvent_t e0 = t->next_event(), e1 = t->next_event();
      if (e0) cudaEventRecord(e0, s);
      // chunked: the leaves of the two resident chunk buffers are read
      // there, the rest from the mapped host copy
      ChunkBufs cb;
      if (t->chunked && !t->point_chunks)
        for (int b = 0; b < 2; ++b)
          if (t->buf_chunk[b] >= 0) {
            CU(cudaStreamWaitEvent(s, t->ev_copied[b], 0));
            cb.buf[b] = t->d_chunk_buf[b];
            cb.lo[b] = t->chunk_leaf[t->buf_chunk[b]];
            cb.hi[b] = t->chunk_leaf[t->buf_chunk[b] + 1];
          }
      CU(launch_tail(D, t->chunked ? t->h_pts : t->d_pts, nxt, n_next,
                     t->state.p, t->qpad.p, t->lst_d.p, t->lst_i.p, K,
                     t->d_ctr, t->sm_count, s, cb));
      if (e1) cudaEventRecord(e1, s);
      if (e0 && e1) t->tail_ev.push_back({e0, e1});
      t->st_tail_queries += n_next;
      t->st_launches += 1;
      break;
    }
    rc = process_round(n_items);
    if (rc != BKD_OK) return rc;
    n_act = n_next;  // an upper bound of every later round's active count
    // rounds queued before the host looks again: many while far from the
    // tail threshold, a few when close to it (a round past the threshold
    // only costs its few queries), one on chunked trees (the host picks
    // the chunks of every round)
    const int batch = t->chunked            ? 1
                      : t->round_batch > 0    ? t->round_batch
                      : n_next > 16 * std::max(tail, 1024) ? 64
                      : n_next > 4 * std::max(tail, 1024)  ? 16
                                                            : 4;
    for (int j = 1; j < batch; ++j) {
      rc = start_round(true);
      if (rc == BKD_OK) rc = process_round(-1);
      if (rc != BKD_OK) return rc;
    }
    rc = start_round(!t->chunked);
    if (rc != BKD_OK) return rc;
  }
  cudaEvent_t x0 = t->next_event();
  if (x0) cudaEventRecord(x0, s);
  CU(launch_recheck(D, m, k, K, t->qpad.p, t->lst_d.p, t->lst_i.p, out_idx,
                    out_dist, t->fb_list.p, t->d_ctr, s));
  CU(cudaMemcpyAsync(t->h_ctr, t->d_ctr, sizeof(Counters),
                     cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  t->st_launches += 1;
  if (t->h_ctr->err & kErrTimeout)
    return fail(BKD_ETIMEOUT, "a leaf-segment copy did not complete");
  if (t->h_ctr->err & kErrBadList)
    return fail(BKD_ECUDA, "internal error: a finished candidate list holds "
                           "an empty entry");
  const int n_fb = t->h_ctr->n_fallback;
  t->st_fallback += n_fb;
  t->st_tail_visits += (double)t->h_ctr->tail_visits;
  t->st_tail_pairs += (double)t->h_ctr->tail_pairs;
  t->st_screen_kept += (double)t->h_ctr->screen_kept;
  t->st_pairs += (double)t->h_ctr->leaf_pairs;
  t->st_leaf_bytes += (double)t->h_ctr->leaf_bytes;
  // rounds processed = every bucketing but the last; screened rounds = all
  // processed rounds but the first
  {
    const Counters& h = *t->h_ctr;
    t->st_visits += (double)(h.rounds_visits - last_visits);
    if (t->precision == 1 && screen_max > 0 &&
        (!t->chunked || t->chunk_screen) &&
        h.rounds_visits > first_visits + last_visits) {
      t->st_screen_visits +=
          (double)(h.rounds_visits - first_visits - last_visits);
      t->st_screen_pairs += (double)(h.rounds_pairs - first_pairs - last_pairs);
      t->st_screen_items += (double)(h.rounds_items - first_items - last_items);
    }
  }
  t->st_screen_bytes += (double)t->h_ctr->screen_bytes;
  t->st_screen_queued += (double)t->h_ctr->screen_queued;
  t->st_screen_overflow += (double)t->h_ctr->screen_overflow;
  t->st_resorted += t->h_ctr->n_resorted;
  if (n_fb > 0) {
    CU(launch_fallback(D, n_fb, t->fb_list.p, k, K, t->qpad.p, t->lst_d.p,
                       out_idx, out_dist, s, t->d_ctr));
    t->st_launches += 1;
    CU(cudaMemcpyAsync(&t->h_ctr->fallback_points,
                       &t->d_ctr->fallback_points, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    t->st_fallback_points += (double)t->h_ctr->fallback_points;
  }
  // chunked trees: what the tail, re-check and fallback kernels read from
  // the mapped (pinned host) leaf structure, point coordinates counted
  if (t->chunked)
    t->st_mapped_bytes +=
        4.0 * Dp *
        ((double)t->h_ctr->tail_mapped_pairs +
         (double)t->h_ctr->n_resorted * k +
         (n_fb > 0 ? (double)t->h_ctr->fallback_points : 0.0));
  cudaEvent_t x1 = t->next_event();
  if (x1) cudaEventRecord(x1, s);
  if (x0 && x1) t->exact_ev.push_back({x0, x1});
  return BKD_OK;
}

}  // namespace

namespace bkd {

namespace {
// Allocations left before the one that is made to fail (0: none fails).
std::atomic<int64_t> g_fail_countdown{0};

bool injected_failure() {
  int64_t c = g_fail_countdown.load();
  while (c > 0) {
    if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
  }
  return false;
}
}  // namespace

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t host_alloc_raw(void** p, size_t bytes, unsigned flags) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaHostAlloc(p, bytes, flags);
}

TreeView view_of(const bkd_tree* t) {
  TreeView v;
  v.device = t->device;
  v.sm_count = t->sm_count;
  v.stream = t->stream;
  v.dev = t->dev;
  v.n_leaves = t->n_leaves;
  v.chunked = t->chunked;
  v.d_pts = t->d_pts;
  v.h_ctr = t->h_ctr;
  v.screen = t->screen;
  v.precision = t->precision;
  v.tail_queries = t->tail_queries;
  v.rescue_rounds = t->rescue_rounds;
  v.defer_queries = t->defer_queries;
  return v;
}

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

}  // namespace bkd

extern "C" {

int bkd_build(const float* P, int64_t n, int d, int height, bkd_tree** out) {
  g_err.clear();
  return build_impl(P, n, d, height, nullptr, 0, out);
}

int bkd_build_with(const float* P, int64_t n, int d, int height,
                   const int64_t* options, int n_options, bkd_tree** out) {
  g_err.clear();
  return build_impl(P, n, d, height, options, n_options, out);
}

int bkd_query(bkd_tree* t, const float* Q, int64_t m, int k, int64_t* out_idx,
              float* out_dist) {
  g_err.clear();
  if (!t) return fail(BKD_EINVAL, "tree is NULL");
  if (m < 0) return fail(BKD_EINVAL, "m must be >= 0");
  if (k < 1 || k > t->dev.n)
    return fail(BKD_EINVAL, "k must be in [1, n] (got %d)", k);
  if (k > BKD_MAX_K)
    return fail(BKD_EUNSUPPORTED, "k = %d exceeds BKD_MAX_K = %d", k,
                BKD_MAX_K);
  if (m > 0 && (!Q || !out_idx || !out_dist))
    return fail(BKD_EINVAL, "Q / out_idx / out_dist is NULL");
  if (m >= (int64_t)1 << 31)
    return fail(BKD_EUNSUPPORTED, "m >= 2^31; slice the query set");
  DeviceGuard guard(t->device);
  reset_stats(t);
  if (m == 0) return BKD_OK;
  const int d = t->dev.d;
  cudaStream_t s = t->stream;
  const PtrKind qk = ptr_kind(Q, t->device), ik = ptr_kind(out_idx, t->device),
                dk = ptr_kind(out_dist, t->device);
  if (qk == kForeignPtr || ik == kForeignPtr || dk == kForeignPtr)
    return fail(BKD_EINVAL, "Q / out_idx / out_dist is device memory of "
                            "another GPU than the tree's (device %d)",
                t->device);
  const bool q_dev = qk == kDevicePtr;
  const bool o_dev = ik == kDevicePtr && dk == kDevicePtr;
  const int64_t slice = t->max_active > 0 ? t->max_active : m;
  CU(t->qdev.ensure(std::min(slice, m) * d));
  if (!o_dev) {
    CU(t->out_idx.ensure(m * k));
    CU(t->out_dist.ensure(m * k));
  }
  for (int64_t q0 = 0; q0 < m; q0 += slice) {
    const int64_t mm = std::min(slice, m - q0);
    CU(cudaMemcpyAsync(t->qdev.p, Q + q0 * d, sizeof(float) * mm * d,
                       q_dev ? cudaMemcpyDeviceToDevice
                             : cudaMemcpyHostToDevice,
                       s));
    int64_t* oi = o_dev ? out_idx + q0 * k : t->out_idx.p + q0 * k;
    float* od = o_dev ? out_dist + q0 * k : t->out_dist.p + q0 * k;
    int rc = search(t, mm, k, oi, od);
    if (rc != BKD_OK) return rc;
  }
  if (!o_dev) {
    CU(cudaMemcpyAsync(out_idx, t->out_idx.p, sizeof(int64_t) * m * k,
                       cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(out_dist, t->out_dist.p, sizeof(float) * m * k,
                       cudaMemcpyDeviceToHost, s));
  }
  CU(cudaStreamSynchronize(s));
  if (t->copy_stream) CU(cudaStreamSynchronize(t->copy_stream));
  collect_timings(t);
  return BKD_OK;
}

int bkd_outlier_scores(bkd_tree* t, int k, float* out_score) {
  g_err.clear();
  if (!t) return fail(BKD_EINVAL, "tree is NULL");
  const int64_t n = t->dev.n;
  if (k < 1 || (int64_t)k + 1 > n)
    return fail(BKD_EINVAL, "k must be in [1, n - 1] (got %d)", k);
  if (k + 1 > BKD_MAX_K)
    return fail(BKD_EUNSUPPORTED, "k + 1 = %d exceeds BKD_MAX_K = %d", k + 1,
                BKD_MAX_K);
  if (!out_score) return fail(BKD_EINVAL, "out_score is NULL");
  DeviceGuard guard(t->device);
  const PtrKind ok = ptr_kind(out_score, t->device);
  if (ok == kForeignPtr)
    return fail(BKD_EINVAL, "out_score is device memory of another GPU");
  reset_stats(t);
  cudaStream_t s = t->stream;
  const int d = t->dev.d, K = k + 1;
  const int64_t slots = t->n_leaves * t->dev.lcap;
  const int64_t slice =
      std::min<int64_t>(n, t->max_active > 0 ? t->max_active : 1 << 24);
  CU(t->inv.ensure(n));
  CU(t->qdev.ensure(slice * d));
  CU(t->out_idx.ensure(slice * K));
  CU(t->out_dist.ensure(slice * K));
  if (ok != kDevicePtr) CU(t->score.ensure(slice));
  // pts / orig: device memory, or mapped pinned host memory (chunked)
  CU(launch_inverse(t->dev.orig, slots, t->inv.p, s));
  for (int64_t i0 = 0; i0 < n; i0 += slice) {
    const int64_t mm = std::min(slice, n - i0);
    CU(launch_gather(t->dev.pts, t->dev.Dp, d, t->inv.p, i0, mm, t->qdev.p,
                     s));
    int rc = search(t, mm, K, t->out_idx.p, t->out_dist.p);
    if (rc != BKD_OK) return rc;
    float* dst = ok == kDevicePtr ? out_score + i0 : t->score.p;
    CU(launch_score(t->out_idx.p, t->out_dist.p, i0, mm, k, dst, s));
    if (ok != kDevicePtr)
      CU(cudaMemcpyAsync(out_score + i0, t->score.p, sizeof(float) * mm,
                         cudaMemcpyDeviceToHost, s));
    t->st_launches += 3;
  }
  CU(cudaStreamSynchronize(s));
  if (t->copy_stream) CU(cudaStreamSynchronize(t->copy_stream));
  collect_timings(t);
  return BKD_OK;
}

int bkd_set_option(bkd_tree* t, int key, int64_t value) {
  g_err.clear();
  if (!t) return fail(BKD_EINVAL, "tree is NULL");
  switch (key) {
    case BKD_OPT_STREAM:
      t->stream = value ? reinterpret_cast<cudaStream_t>(value) : t->own_stream;
      return BKD_OK;
    case BKD_OPT_MAX_ACTIVE:
      if (value < 0 || value >= ((int64_t)1 << 31))
        return fail(BKD_EINVAL, "max active out of range");
      t->max_active = (int)value;
      return BKD_OK;
    case BKD_OPT_PRECISION:
      if (value != 0 && value != 1)
        return fail(BKD_EINVAL, "precision must be 0 or 1");
      if (value == 1 && !t->screen.on())
        return fail(BKD_EINVAL,
                    "the tree was built without BF16 screen data (pass "
                    "BKD_OPT_PRECISION=1 to bkd_build_with)");
      t->precision = (int)value;
      return BKD_OK;
    case BKD_OPT_TAIL_QUERIES:
      if (value < -1 || value >= ((int64_t)1 << 31))
        return fail(BKD_EINVAL, "tail query count out of range");
      t->tail_queries = (int)value;
      return BKD_OK;
    case BKD_OPT_SCREEN_TILE: {
      // the warp kernel: 8-query column blocks, one query per lane; the
      // tcgen05 kernel: the MMA's N in steps of 16
      const int step = t->screen.kind == 0 ? 8 : 16;
      const int top = screen_tile_of(t->screen.kind);
      if (value < step || value > top || value % step != 0)
        return fail(BKD_EINVAL,
                    "screen tile must be %d..%d, a multiple of %d", step, top,
                    step);
      t->screen_tile = (int)value;
      return BKD_OK;
    }
    case BKD_OPT_RESCUE_ROUNDS:
      if (value < 0 || value >= ((int64_t)1 << 31))
        return fail(BKD_EINVAL, "rescue rounds out of range");
      t->rescue_rounds = (int)value;
      return BKD_OK;
    case BKD_OPT_DEFER_QUERIES:
      if (value < 0 || value > 4096)
        return fail(BKD_EINVAL, "deferral threshold must be 0..4096");
      t->defer_queries = (int)value;
      return BKD_OK;
    case BKD_OPT_SCREEN_KERNEL:
      if (value != 0 && value != 1)
        return fail(BKD_EINVAL, "screen kernel must be 0 or 1");
      if (!t->screen.has((int)value))
        return fail(BKD_EINVAL,
                    "the tree holds no screen data for kernel %lld (build "
                    "with BKD_OPT_PRECISION=1 and BKD_OPT_SCREEN_KERNEL=%lld "
                    "or 2)",
                    (long long)value, (long long)value);
      if (t->screen.kind != (int)value) {
        t->screen.kind = (int)value;
        t->screen_tile = screen_tile_of(t->screen.kind);
      }
      return BKD_OK;
    case BKD_OPT_ROUND_BATCH:
      if (value < 0 || value > 64)
        return fail(BKD_EINVAL, "round batch must be 0..64");
      t->round_batch = (int)value;
      return BKD_OK;
    case BKD_OPT_SCREEN_CTAS:
      if (value < 0 || value > 3)
        return fail(BKD_EINVAL, "screen CTAs per SM must be 0..3");
      t->screen_ctas = (int)value;
      return BKD_OK;
    case BKD_OPT_DEVICE_MEM_CAP:
    case BKD_OPT_CHUNKS:
    case BKD_OPT_POINT_CHUNKS:
      return fail(BKD_EINVAL, "option %d applies at build only", key);
    default:
      return fail(BKD_EINVAL, "unknown option %d", key);
  }
}

int bkd_get_stat(const bkd_tree* t, int key, double* value) {
  g_err.clear();
  if (!t || !value) return fail(BKD_EINVAL, "NULL argument");
  switch (key) {
    case BKD_STAT_ROUNDS: *value = t->st_rounds; break;
    case BKD_STAT_LEAF_VISITS: *value = t->st_visits; break;
    case BKD_STAT_PAIRS: *value = t->st_pairs; break;
    case BKD_STAT_RESORTED: *value = t->st_resorted; break;
    case BKD_STAT_FALLBACK: *value = t->st_fallback; break;
    case BKD_STAT_LEAF_KERNEL_MS: *value = t->st_leaf_ms; break;
    case BKD_STAT_CHUNK_BYTES: *value = t->st_chunk_bytes; break;
    case BKD_STAT_COPY_MS: *value = t->st_copy_ms; break;
    case BKD_STAT_LEAF_LAUNCHES: *value = t->st_leaf_launches; break;
    case BKD_STAT_KERNEL_LAUNCHES: *value = t->st_launches; break;
    case BKD_STAT_TAIL_QUERIES: *value = t->st_tail_queries; break;
    case BKD_STAT_TAIL_VISITS: *value = t->st_tail_visits; break;
    case BKD_STAT_TAIL_PAIRS: *value = t->st_tail_pairs; break;
    case BKD_STAT_TAIL_MS: *value = t->st_tail_ms; break;
    case BKD_STAT_SCREEN_KEPT: *value = t->st_screen_kept; break;
    case BKD_STAT_SCREEN_PAIRS: *value = t->st_screen_pairs; break;
    case BKD_STAT_SCREEN_MS: *value = t->st_screen_ms; break;
    case BKD_STAT_SCREEN_ITEMS: *value = t->st_screen_items; break;
    case BKD_STAT_SCREEN_VISITS: *value = t->st_screen_visits; break;
    case BKD_STAT_FIND_MS: *value = t->st_find_ms; break;
    case BKD_STAT_BUCKET_MS: *value = t->st_bucket_ms; break;
    case BKD_STAT_EXACT_MS: *value = t->st_exact_ms; break;
    case BKD_STAT_CHUNK_VISITS: *value = t->st_chunk_visits; break;
    case BKD_STAT_SCREEN_BYTES: *value = t->st_screen_bytes; break;
    case BKD_STAT_LEAF_BYTES: *value = t->st_leaf_bytes; break;
    case BKD_STAT_HOST_SYNCS: *value = t->st_host_syncs; break;
    case BKD_STAT_FALLBACK_POINTS: *value = t->st_fallback_points; break;
    case BKD_STAT_MAPPED_BYTES: *value = t->st_mapped_bytes; break;
    case BKD_STAT_SCREEN_QUEUED: *value = t->st_screen_queued; break;
    case BKD_STAT_SCREEN_OVERFLOW: *value = t->st_screen_overflow; break;
    default: return fail(BKD_EINVAL, "unknown stat %d", key);
  }
  return BKD_OK;
}

int bkd_tree_shape(const bkd_tree* t, int64_t* n, int* d, int* height,
                   int* chunked, int* chunks) {
  g_err.clear();
  if (!t) return fail(BKD_EINVAL, "tree is NULL");
  if (n) *n = t->dev.n;
  if (d) *d = t->dev.d;
  if (height) *height = t->dev.h;
  if (chunked) *chunked = t->chunked ? 1 : 0;
  if (chunks) *chunks = t->n_chunks;
  return BKD_OK;
}

int bkd_export_tree(const bkd_tree* t, float* split, int64_t* leaf_lo,
                    int64_t* perm) {
  g_err.clear();
  if (!t) return fail(BKD_EINVAL, "tree is NULL");
  const int64_t L = t->n_leaves;
  if (split && L > 1) std::memcpy(split, t->host.split, sizeof(float) * (L - 1));
  if (leaf_lo) std::memcpy(leaf_lo, t->host.leaf_lo, sizeof(int64_t) * (L + 1));
  if (perm) std::memcpy(perm, t->host.perm, sizeof(int64_t) * t->dev.n);
  return BKD_OK;
}

void bkd_free(bkd_tree* t) { release(t); }

int bkd_test_fail_alloc(int64_t nth) {
  g_err.clear();
  if (nth < 0) return fail(BKD_EINVAL, "nth must be >= 0");
  bkd::g_fail_countdown.store(nth);
  return BKD_OK;
}

const char* bkd_last_error(void) { return g_err.c_str(); }

}  // extern "C"
