// k_traverse.cu -- query initialisation and FindLeafBatch (Algorithm 1).
//
// FindLeafBatch continues each query's "implicit tree traversal" (Sec. 2.4)
// to the next leaf it has to visit, or reports -1 once the traversal has
// reached the root twice.  The traversal is the classical k-d tree search of
// Sec. 2.3: walk down to the cell containing q; on the way back up, visit the
// far child of a node iff it could still hold a better candidate, otherwise
// prune.
//
// The traversal step itself (stackless, exact bounding-box pruning) is
// next_leaf() in traverse.cuh, shared with the tail and fallback kernels.
#include "bkd_internal.h"
#include "traverse.cuh"

namespace bkd {
namespace {

__global__ void init_kernel(const float* __restrict__ Q, int64_t m, int d,
                            int Dp, float* __restrict__ qpad,
                            float* __restrict__ lst_d,
                            uint32_t* __restrict__ lst_i, int K,
                            int32_t* __restrict__ state,
                            uint32_t* __restrict__ act, Counters* ctr) {
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
  state[q] = kStart;
  act[q] = (uint32_t)q;
  if (bad) atomicOr(&ctr->err, kErrNonFinite);
}

__global__ void find_leaf_kernel(DevTree t, const float* __restrict__ qpad,
                                 const uint32_t* __restrict__ act, int n_act,
                                 int32_t* __restrict__ state,
                                 const float* __restrict__ lst_d, int K,
                                 int32_t* __restrict__ leaf_of) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= n_act) return;
  const uint32_t q = act[pos];
  const float* qp = qpad + (size_t)q * t.Dp;
  const int node = state[q];
  const float bound = node == kStart ? __int_as_float(0x7f800000)
                                     : lst_d[(size_t)q * K + (K - 1)];
  const int next = next_leaf<F32Bound>(t, qp, node, bound);
  state[q] = next;
  leaf_of[pos] = next == kDone ? -1 : next - ((1 << t.h) - 1);
}

// ------------------------------------------------------------- bucketing
// Buffer insertion of Algorithm 1 as a counting sort by leaf id: histogram,
// exclusive scan (also of per-leaf work items of kTileQ queries), scatter.
// The order of queries inside a leaf's buffer is irrelevant to the results.

__global__ void hist_kernel(const int32_t* __restrict__ leaf_of, int n,
                            int32_t* __restrict__ cnt) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= n) return;
  const int l = leaf_of[pos];
  if (l >= 0) atomicAdd(cnt + l, 1);
}

constexpr int kScanThreads = 1024;

// One block: exclusive scans of cnt (-> off) and of ceil(cnt / kTileQ)
// (-> toff), the item list, and the round totals.
__global__ void __launch_bounds__(kScanThreads)
    scan_kernel(const int32_t* __restrict__ cnt, int L,
                const int32_t* __restrict__ leaf_cnt,
                int32_t* __restrict__ off, int32_t* __restrict__ toff,
                Item* __restrict__ items, Counters* ctr) {
  __shared__ int32_t s_q[kScanThreads / 32], s_t[kScanThreads / 32];
  __shared__ unsigned long long s_p[kScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (L + kScanThreads - 1) / kScanThreads;
  const int lo = min(L, tid * per), hi = min(L, lo + per);
  int32_t sq = 0, st = 0;
  unsigned long long sp = 0;
  for (int l = lo; l < hi; ++l) {
    const int c = cnt[l];
    sq += c;
    st += (c + kTileQ - 1) / kTileQ;
    sp += (unsigned long long)c * (unsigned long long)leaf_cnt[l];
  }
  // inclusive warp scans
  int32_t iq = sq, it = st;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t a = __shfl_up_sync(0xffffffffu, iq, o);
    const int32_t b = __shfl_up_sync(0xffffffffu, it, o);
    if (lane >= o) {
      iq += a;
      it += b;
    }
  }
  unsigned long long wp = sp;
  for (int o = 16; o > 0; o >>= 1) wp += __shfl_down_sync(0xffffffffu, wp, o);
  if (lane == 31) {
    s_q[warp] = iq;
    s_t[warp] = it;
  }
  if (lane == 0) s_p[warp] = wp;
  __syncthreads();
  if (warp == 0) {
    int32_t a = s_q[lane], b = s_t[lane];
    unsigned long long p = s_p[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t x = __shfl_up_sync(0xffffffffu, a, o);
      const int32_t y = __shfl_up_sync(0xffffffffu, b, o);
      if (lane >= o) {
        a += x;
        b += y;
      }
    }
    for (int o = 16; o > 0; o >>= 1) p += __shfl_down_sync(0xffffffffu, p, o);
    s_q[lane] = a;
    s_t[lane] = b;
    if (lane == 0) s_p[0] = p;
  }
  __syncthreads();
  int32_t bq = (warp > 0 ? s_q[warp - 1] : 0) + iq - sq;
  int32_t bt = (warp > 0 ? s_t[warp - 1] : 0) + it - st;
  for (int l = lo; l < hi; ++l) {
    const int c = cnt[l];
    const int nt = (c + kTileQ - 1) / kTileQ;
    off[l] = bq;
    toff[l] = bt;
    for (int j = 0; j < nt; ++j) {
      Item w;
      w.leaf = l;
      w.start = bq + j * kTileQ;
      w.count = min(kTileQ, c - j * kTileQ);
      w.pad = 0;
      items[bt + j] = w;
    }
    bq += c;
    bt += nt;
  }
  if (tid == kScanThreads - 1) {
    off[L] = s_q[31];
    toff[L] = s_t[31];
    ctr->n_next = s_q[31];
    ctr->n_items = s_t[31];
    ctr->pairs = s_p[0];
  }
}

__global__ void scatter_kernel(const int32_t* __restrict__ leaf_of,
                               const uint32_t* __restrict__ act, int n,
                               const int32_t* __restrict__ off,
                               int32_t* __restrict__ cursor,
                               uint32_t* __restrict__ next) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= n) return;
  const int l = leaf_of[pos];
  if (l < 0) return;
  next[off[l] + atomicAdd(cursor + l, 1)] = act[pos];
}

__global__ void chunk_items_kernel(const int32_t* __restrict__ toff,
                                   const int32_t* __restrict__ chunk_leaf,
                                   int n_chunks, int32_t* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c <= n_chunks) out[c] = toff[chunk_leaf[c]];
}

inline int blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_init(const float* Q, int64_t m, int d, int Dp, float* qpad,
                        float* lst_d, uint32_t* lst_i, int K, int32_t* state,
                        uint32_t* act, Counters* ctr, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  init_kernel<<<blocks(m, 256), 256, 0, s>>>(Q, m, d, Dp, qpad, lst_d, lst_i,
                                             K, state, act, ctr);
  return cudaGetLastError();
}

cudaError_t launch_find_leaf(const DevTree& t, const float* qpad,
                             const uint32_t* act, int n_act, int32_t* state,
                             const float* lst_d, int K, int32_t* leaf_of,
                             cudaStream_t s) {
  if (n_act == 0) return cudaSuccess;
  find_leaf_kernel<<<blocks(n_act, 256), 256, 0, s>>>(t, qpad, act, n_act,
                                                      state, lst_d, K, leaf_of);
  return cudaGetLastError();
}

cudaError_t launch_bucket(const int32_t* leaf_of, const uint32_t* act,
                          int n_act, int n_leaves, const int32_t* leaf_cnt,
                          int32_t* cnt, int32_t* off, int32_t* cursor,
                          int32_t* toff, Item* items, uint32_t* next,
                          Counters* ctr, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n_leaves, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * n_leaves, s);
  if (e != cudaSuccess) return e;
  if (n_act > 0) hist_kernel<<<blocks(n_act, 256), 256, 0, s>>>(leaf_of, n_act, cnt);
  scan_kernel<<<1, kScanThreads, 0, s>>>(cnt, n_leaves, leaf_cnt, off, toff,
                                         items, ctr);
  if (n_act > 0)
    scatter_kernel<<<blocks(n_act, 256), 256, 0, s>>>(leaf_of, act, n_act, off,
                                                      cursor, next);
  return cudaGetLastError();
}

cudaError_t launch_chunk_items(const int32_t* toff, const int32_t* chunk_leaf,
                               int n_chunks, int32_t* chunk_item,
                               cudaStream_t s) {
  chunk_items_kernel<<<blocks(n_chunks + 1, 128), 128, 0, s>>>(
      toff, chunk_leaf, n_chunks, chunk_item);
  return cudaGetLastError();
}

}  // namespace bkd
