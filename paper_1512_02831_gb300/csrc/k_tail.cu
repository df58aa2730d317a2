// k_tail.cu -- finishing the last active queries without further rounds.
//
// LazySearch advances every active query by one leaf per round (Algorithm 1),
// so the number of rounds equals the largest number of leaves any single
// query visits, while the number of active queries -- and with it the work
// per round -- decays.  Once few queries remain, each further round is mostly
// fixed cost (traversal, bucketing, a launch over a few buffers of one query
// each).  This kernel takes the remaining queries and runs each one's
// traversal to the end: one warp per query, the same traversal step as
// FindLeafBatch (traverse.cuh), the leaf's quads split across the lanes, and
// the same float32 distance chain as the leaf kernel.  The candidate list is
// spread over the warp (lane j holds entry j) and a candidate is inserted iff
// its distance is strictly below the last entry, so the list ends with the
// same multiset of k+1 smallest float32 distances as the round-by-round path.
// Lists of up to 64 entries (k <= 63) take two entries per lane.
#include "bkd.h"
#include "k_leaf.cuh"
#include "traverse.cuh"

namespace bkd {
namespace {

constexpr int kTailWarps = 4;

// The candidate list of K <= 64 entries spread over the warp: lane j holds
// entry j and, when TWO, entry 32 + j.  Inserting (cd, id) below the bound
// moves every entry from its sorted position on up by one place.
template <bool TWO>
struct WarpList {
  float d0 = __builtin_huge_valf(), d1 = __builtin_huge_valf();
  uint32_t i0 = kNoSlot, i1 = kNoSlot;
  __device__ void load(const float* ld, const uint32_t* li, int K, int lane) {
    if (lane < K) {
      d0 = ld[lane];
      i0 = li[lane];
    }
    if (TWO && 32 + lane < K) {
      d1 = ld[32 + lane];
      i1 = li[32 + lane];
    }
  }
  __device__ void store(float* ld, uint32_t* li, int K, int lane) const {
    if (lane < K) {
      ld[lane] = d0;
      li[lane] = i0;
    }
    if (TWO && 32 + lane < K) {
      ld[32 + lane] = d1;
      li[32 + lane] = i1;
    }
  }
  __device__ float bound(int K) const {
    const unsigned full = 0xffffffffu;
    if (!TWO || K <= 32) return __shfl_sync(full, d0, K - 1);
    return __shfl_sync(full, d1, K - 33);
  }
  // requires cd below the bound (warp-uniform)
  __device__ void insert(float cd, uint32_t id, int K, int lane) {
    const unsigned full = 0xffffffffu;
    int pos = __popc(__ballot_sync(full, lane < K && d0 <= cd));
    if (TWO) pos += __popc(__ballot_sync(full, 32 + lane < K && d1 <= cd));
    const float u0 = __shfl_up_sync(full, d0, 1);
    const uint32_t v0 = __shfl_up_sync(full, i0, 1);
    if (TWO) {
      const float u1 = __shfl_up_sync(full, d1, 1);
      const uint32_t v1 = __shfl_up_sync(full, i1, 1);
      const float c31 = __shfl_sync(full, d0, 31);
      const uint32_t j31 = __shfl_sync(full, i0, 31);
      const int k1 = 32 + lane;
      if (k1 > pos) {
        d1 = lane ? u1 : c31;
        i1 = lane ? v1 : j31;
      } else if (k1 == pos) {
        d1 = cd;
        i1 = id;
      }
    }
    if (lane > pos) {
      d0 = u0;
      i0 = v0;
    } else if (lane == pos) {
      d0 = cd;
      i0 = id;
    }
  }
};

template <int D, bool TWO>
__global__ void __launch_bounds__(kTailWarps * 32)
    tail_kernel(DevTree t, const float4* __restrict__ pts,
                const uint32_t* __restrict__ act, int n_act,
                uint64_t* __restrict__ state, const float* __restrict__ qpad,
                float* __restrict__ lst_d, uint32_t* __restrict__ lst_i, int K,
                Counters* ctr, ChunkBufs cb, bool after_scanned) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const int first_leaf = (1 << t.h) - 1;
  const int64_t qpl = t.lcap >> 2;
  unsigned long long pairs = 0, visits = 0, mapped = 0;
  for (int w = blockIdx.x * kTailWarps + (threadIdx.x >> 5); w < n_act;
       w += gridDim.x * kTailWarps) {
    const uint32_t q = act[w];
    const float* qp = qpad + (size_t)q * D;
    uint64_t qq[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float x = qp[i];
      qq[i] = pk2(x, x);
    }
    WarpList<TWO> L;
    L.load(lst_d + (size_t)q * K, lst_i + (size_t)q * K, K, lane);
    float bound = L.bound(K);
    F32Bound<D> bx;
    bx.load(qp);
    // state holds the query's pending leaf: scan it, then walk on
    const uint64_t st = state[q];
    int node = state_node(st);
    uint32_t mask = state_mask(st);
    if (node == kStart ||
        (after_scanned && !(t.q_wait && t.q_wait[q])))
      node = next_leaf(t, bx, qp, node, mask, bound);
    for (; node != kDone; node = next_leaf(t, bx, qp, node, mask, bound)) {
      const int leaf = node - first_leaf;
      const int np = t.leaf_cnt[leaf];
      const int nq = (np + 3) >> 2;
      // the leaf in a device chunk buffer if one holds it, else at pts
      const float4* lq;
      if (leaf >= cb.lo[0] && leaf < cb.hi[0]) {
        lq = reinterpret_cast<const float4*>(cb.buf[0]) +
             (int64_t)(leaf - cb.lo[0]) * qpl * D;
      } else if (leaf >= cb.lo[1] && leaf < cb.hi[1]) {
        lq = reinterpret_cast<const float4*>(cb.buf[1]) +
             (int64_t)(leaf - cb.lo[1]) * qpl * D;
      } else {
        lq = pts + (int64_t)leaf * qpl * D;
        mapped += (unsigned long long)np;
      }
      const uint32_t slot0 = (uint32_t)((int64_t)leaf * t.lcap);
      ++visits;
      pairs += (unsigned long long)np;
      // up to 16 dimensions, the quads of the next 32-quad chunk are loaded
      // while this one is scored (one warp on one query: a visit is
      // latency-bound); above, the registers would not hold two chunks
      constexpr bool kPipe = D <= 16;
      float4 nb[kPipe ? D : 1];
      if constexpr (kPipe) {
#pragma unroll
        for (int i = 0; i < D; ++i)
          nb[i] = lane < nq ? lq[(int64_t)lane * D + i]
                            : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      for (int g0 = 0; g0 < nq; g0 += 32) {
        const int g = g0 + lane;
        float4 cb[D];
        if constexpr (kPipe) {
#pragma unroll
          for (int i = 0; i < D; ++i) cb[i] = nb[i];
          if (g0 + 32 < nq) {
#pragma unroll
            for (int i = 0; i < D; ++i)
              nb[i] = g + 32 < nq ? lq[(int64_t)(g + 32) * D + i]
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        } else {
#pragma unroll
          for (int i = 0; i < D; ++i)
            cb[i] = g < nq ? lq[(int64_t)g * D + i]
                           : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float e[4] = {__int_as_float(0x7f800000), __int_as_float(0x7f800000),
                      __int_as_float(0x7f800000), __int_as_float(0x7f800000)};
        if (g < nq) quad_dist<D>(cb, qq, e[0], e[1], e[2], e[3]);
        unsigned cand = __ballot_sync(
            full, fminf(fminf(e[0], e[1]), fminf(e[2], e[3])) < bound);
        while (cand) {
          const int src = __ffs(cand) - 1;
          cand &= cand - 1;
          const uint32_t id = slot0 + (uint32_t)(g0 + src) * 4u;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float cd = __shfl_sync(full, e[j], src);
            if (cd < bound) {  // warp-uniform
              L.insert(cd, id + j, K, lane);
              bound = L.bound(K);
            }
          }
        }
      }
    }
    L.store(lst_d + (size_t)q * K, lst_i + (size_t)q * K, K, lane);
    if (lane == 0) state[q] = trav_state(kDone, 0u);
  }
  if (lane == 0 && visits) {
    atomicAdd(&ctr->tail_pairs, pairs);
    atomicAdd(&ctr->tail_visits, visits);
    if (mapped) atomicAdd(&ctr->tail_mapped_pairs, mapped);
  }
}

#define BKD_TAIL_CASE(DIM)                                                   \
  case DIM:                                                                  \
    if (K <= 32)                                                             \
      tail_kernel<DIM, false><<<grid, kTailWarps * 32, 0, s>>>(              \
          t, reinterpret_cast<const float4*>(pts), act, n_act, state, qpad,  \
          lst_d, lst_i, K, ctr, cb, after_scanned);                          \
    else                                                                     \
      tail_kernel<DIM, true><<<grid, kTailWarps * 32, 0, s>>>(               \
          t, reinterpret_cast<const float4*>(pts), act, n_act, state, qpad,  \
          lst_d, lst_i, K, ctr, cb, after_scanned);                          \
    return cudaGetLastError();

}  // namespace

cudaError_t launch_tail(const DevTree& t, const float* pts,
                        const uint32_t* act, int n_act, uint64_t* state,
                        const float* qpad, float* lst_d, uint32_t* lst_i,
                        int K, Counters* ctr, int sm_count, cudaStream_t s,
                        const ChunkBufs& cb, bool after_scanned) {
  if (n_act <= 0) return cudaSuccess;
  if (K < 1 || K > 64) return cudaErrorInvalidValue;
  const int grid = std::min((n_act + kTailWarps - 1) / kTailWarps,
                            sm_count * 16);
  switch (t.Dp) { BKD_LEAF_DIMS(BKD_TAIL_CASE) default: break; }
  return cudaErrorInvalidValue;
}

}  // namespace bkd
