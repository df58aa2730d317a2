// static_query.cu -- bkd_query_static: a query entry point that allocates
// nothing.
//
// Some callers cannot call cudaMalloc while they answer queries: a serving
// process whose device memory is entirely owned by its own pool allocator
// (a stray cudaMalloc fails or fragments the pool), or a latency-critical
// loop that cannot afford cudaMalloc / cudaFree (cudaFree synchronises the
// whole device and stalls every other stream).  bkd_query allocates its
// workspace on first use and grows it with the query count; this entry point
// instead runs the same kernels on a fixed scratch area that lives in a
// file-scope __device__ array, so a call performs no allocation at all.
//
// The array is static device memory of the library: every GPU that loads the
// library holds BKD_STATIC_SCRATCH_BYTES of it until the process exits.  Host
// code cannot use the array's name as a device address (in host code the name
// is a host-side stand-in), so the first call on each device asks the runtime
// for its device address with cudaGetSymbolAddress, with that device current,
// and remembers it.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "bkd.h"
#include "bkd_internal.h"

namespace bkd {
namespace {

constexpr int64_t kAlign = 256;
constexpr int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

constexpr int64_t kQ = BKD_STATIC_MAX_QUERIES;
constexpr int64_t kL = (int64_t)1 << BKD_STATIC_MAX_HEIGHT;
constexpr int64_t kKc = BKD_MAX_K + 1;   // largest list length k + 1
constexpr int64_t kDc = BKD_MAX_DIM;     // largest compiled dimension

// Byte offsets of the pieces carved out of the scratch array.
constexpr int64_t kOffQpad = 0;
constexpr int64_t kOffLstD = kOffQpad + align_up(kQ * kDc * 4);
constexpr int64_t kOffLstI = kOffLstD + align_up(kQ * kKc * 4);
constexpr int64_t kOffState = kOffLstI + align_up(kQ * kKc * 4);
constexpr int64_t kOffActA = kOffState + align_up(kQ * 8);
constexpr int64_t kOffActB = kOffActA + align_up(kQ * 4);
constexpr int64_t kOffPlaced = kOffActB + align_up(kQ * 4);
constexpr int64_t kOffFb = kOffPlaced + align_up(kQ * 8);
constexpr int64_t kOffCnt = kOffFb + align_up(kQ * 4);
constexpr int64_t kOffCursor = kOffCnt + align_up(kL * 4);
constexpr int64_t kOffOff = kOffCursor + align_up(kL * 4);
constexpr int64_t kOffToff = kOffOff + align_up((kL + 1) * 4);
constexpr int64_t kOffItems = kOffToff + align_up((kL + 1) * 4);
constexpr int64_t kOffCtr =
    kOffItems + align_up((kQ / kPipeTile + kL + 1) * (int64_t)sizeof(Item));
constexpr int64_t kScratchBytes = kOffCtr + align_up(sizeof(Counters));
static_assert(kScratchBytes <= BKD_STATIC_SCRATCH_BYTES,
              "BKD_STATIC_SCRATCH_BYTES too small for the static layout");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
char* g_scratch_addr[kMaxDevices] = {};

}  // namespace
}  // namespace bkd

// The scratch area shared by every bkd_query_static call on a device.
static __device__ __align__(256) unsigned char
    g_static_scratch[BKD_STATIC_SCRATCH_BYTES];

namespace bkd {
namespace {

// Device address of g_static_scratch on `device` (which must be current).
int scratch_address(int device, char** out) {
  if (device < 0 || device >= kMaxDevices)
    return set_error(BKD_EUNSUPPORTED, "device ordinal %d out of range",
                     device);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return set_error(BKD_ECUDA,
                       "cudaGetSymbolAddress of the static scratch failed: %s",
                       cudaGetErrorString(e));
    g_scratch_addr[device] = static_cast<char*>(p);
  }
  *out = g_scratch_addr[device];
  return BKD_OK;
}

// True for device memory the tree's GPU can use: its own, or managed.
// Host memory, and device memory of another GPU (which this GPU's kernels
// could not read without peer access), are refused.
bool on_device(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeManaged ||
         (a.type == cudaMemoryTypeDevice && a.device == device);
}

#define SQ_CU(call)                                                     \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess)                                              \
      return set_error(BKD_ECUDA, "%s failed: %s", #call,               \
                       cudaGetErrorString(e_));                         \
  } while (0)

// LazySearch over the static scratch: the same kernels and the same round
// structure as bkd_query's resident path, without workspace allocation,
// timing events or query slicing.
int run_static(const TreeView& v, char* base, const float* Q, int64_t m, int k,
               int64_t* out_idx, float* out_dist) {
  const int K = k + 1;
  const int cap = list_capacity(K);
  const DevTree& D = v.dev;
  cudaStream_t s = v.stream;
  float* qpad = reinterpret_cast<float*>(base + kOffQpad);
  float* lst_d = reinterpret_cast<float*>(base + kOffLstD);
  uint32_t* lst_i = reinterpret_cast<uint32_t*>(base + kOffLstI);
  uint64_t* state = reinterpret_cast<uint64_t*>(base + kOffState);
  uint32_t* act = reinterpret_cast<uint32_t*>(base + kOffActA);
  uint32_t* nxt = reinterpret_cast<uint32_t*>(base + kOffActB);
  int2* placed = reinterpret_cast<int2*>(base + kOffPlaced);
  uint32_t* fb = reinterpret_cast<uint32_t*>(base + kOffFb);
  int32_t* cnt = reinterpret_cast<int32_t*>(base + kOffCnt);
  int32_t* cursor = reinterpret_cast<int32_t*>(base + kOffCursor);
  int32_t* off = reinterpret_cast<int32_t*>(base + kOffOff);
  int32_t* toff = reinterpret_cast<int32_t*>(base + kOffToff);
  Item* items = reinterpret_cast<Item*>(base + kOffItems);
  Counters* ctr = reinterpret_cast<Counters*>(base + kOffCtr);
  Counters* h = v.h_ctr;

  // The counters keep the previous call's values: clear them.  Everything
  // else is fully written before it is read (init writes lists, state and the
  // active list; every round clears cnt before FindLeafBatch).
  SQ_CU(cudaMemsetAsync(ctr, 0, sizeof(Counters), s));
  SQ_CU(launch_init(Q, m, D.d, D.Dp, qpad, lst_d, lst_i, K, state, act, 0u, ctr,
                    s));
  const int grid_max = leaf_kernel_grid(D.Dp, cap, v.sm_count);
  int n_act = (int)m;
  for (;;) {
    SQ_CU(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * v.n_leaves, s));
    SQ_CU(launch_find_leaf(D, qpad, act, n_act, state, lst_d, K, placed,
                           cnt, s));
    SQ_CU(launch_bucket(placed, act, n_act, (int)v.n_leaves, kPipeTile,
                        D.leaf_cnt, cnt, off, cursor, toff, items, nxt, ctr,
                        s));
    SQ_CU(cudaMemcpyAsync(h, ctr, sizeof(Counters), cudaMemcpyDeviceToHost,
                          s));
    SQ_CU(cudaStreamSynchronize(s));
    if (h->err & kErrNonFinite)
      return set_error(BKD_EINVAL,
                       "Q holds a non-finite or |x| >= 2^60 value");
    if (h->err & kErrTimeout)
      return set_error(BKD_ETIMEOUT, "a leaf-segment copy did not complete");
    const int n_next = h->n_next, n_items = h->n_items;
    if (n_next == 0) break;
    SQ_CU(launch_leaf(D, cap, items, 0, n_items, ctr, v.d_pts, 0, nxt, qpad,
                      lst_d, lst_i, K, std::min(grid_max, n_items), s));
    std::swap(act, nxt);
    n_act = n_next;
  }
  SQ_CU(launch_recheck(D, m, k, K, qpad, lst_d, lst_i, out_idx, out_dist, fb,
                       ctr, s));
  SQ_CU(cudaMemcpyAsync(h, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
  SQ_CU(cudaStreamSynchronize(s));
  if (h->err & kErrTimeout)
    return set_error(BKD_ETIMEOUT, "a leaf-segment copy did not complete");
  if (h->err & kErrBadList)
    return set_error(BKD_ECUDA, "internal error: a finished candidate list "
                                "holds an empty entry");
  if (h->n_fallback > 0)
    SQ_CU(launch_fallback(D, h->n_fallback, fb, k, K, qpad, lst_d, out_idx,
                          out_dist, s));
  SQ_CU(cudaStreamSynchronize(s));
  return BKD_OK;
}

}  // namespace
}  // namespace bkd

extern "C" int bkd_query_static(bkd_tree* t, const float* Q, int64_t m, int k,
                                int64_t* out_idx, float* out_dist) {
  using namespace bkd;
  set_error(BKD_OK, "");
  if (!t) return set_error(BKD_EINVAL, "tree is NULL");
  const TreeView v = view_of(t);
  if (m < 0) return set_error(BKD_EINVAL, "m must be >= 0");
  if (m > BKD_STATIC_MAX_QUERIES)
    return set_error(BKD_EINVAL,
                     "bkd_query_static takes at most %d queries per call "
                     "(got %lld); use bkd_query or split the call",
                     BKD_STATIC_MAX_QUERIES, (long long)m);
  if (k < 1 || k > v.dev.n)
    return set_error(BKD_EINVAL, "k must be in [1, n] (got %d)", k);
  if (k > BKD_MAX_K)
    return set_error(BKD_EUNSUPPORTED, "k = %d exceeds BKD_MAX_K = %d", k,
                     BKD_MAX_K);
  if (v.dev.h > BKD_STATIC_MAX_HEIGHT)
    return set_error(BKD_EINVAL,
                     "bkd_query_static needs a tree of height <= %d (got %d)",
                     BKD_STATIC_MAX_HEIGHT, v.dev.h);
  if (v.chunked || !v.d_pts)
    return set_error(BKD_EUNSUPPORTED,
                     "bkd_query_static needs a tree resident in device "
                     "memory (this tree is chunked)");
  if (m == 0) return BKD_OK;
  if (!Q || !out_idx || !out_dist)
    return set_error(BKD_EINVAL, "Q / out_idx / out_dist is NULL");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess)
    return set_error(BKD_ECUDA, "cudaGetDevice failed");
  if (prev != v.device && cudaSetDevice(v.device) != cudaSuccess)
    return set_error(BKD_ECUDA, "cudaSetDevice(%d) failed", v.device);
  int rc = BKD_OK;
  if (!on_device(Q, v.device) || !on_device(out_idx, v.device) ||
      !on_device(out_dist, v.device)) {
    rc = set_error(BKD_EINVAL,
                   "bkd_query_static takes device pointers only (Q, out_idx, "
                   "out_dist), on the tree's GPU (device %d)", v.device);
  } else {
    char* base = nullptr;
    rc = scratch_address(v.device, &base);
    if (rc == BKD_OK) rc = run_static(v, base, Q, m, k, out_idx, out_dist);
  }
  if (prev != v.device) cudaSetDevice(prev);
  return rc;
}
