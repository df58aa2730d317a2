// k_leaf.cuh -- ProcessAllBuffers: leaf brute force with the k-best merge
// fused in (Algorithm 1; Sec. 3.2: every buffered query of a leaf is
// compared with every reference point of that leaf).
//
// One 64-thread CTA takes one work item at a time: up to 64 buffered queries
// of one leaf, one query per thread.  Each thread holds its query's
// coordinates and sorted candidate list in registers and streams over the
// leaf's quads, which arrive in shared memory through a two-buffer TMA
// pipeline and are read with warp-broadcast float4 loads.
//
// Distance arithmetic (float32, round-to-nearest, no reassociation):
//     e = fl(fl(q_0 - x_0)^2);  e = fma(fl(q_i - x_i), fl(q_i - x_i), e), i=1..D-1
// evaluated two points at a time with the packed sub/mul/fma.rn.f32x2
// instructions, which round each lane exactly like the scalar forms.  The
// traversal's exact-pruning argument depends on this exact sequence.
//
// Candidate list: KT sorted (distance, slot) pairs; the first KT - K entries
// are -1 sentinels that never move, so the list behaves as a K = k+1 list
// whose bound sits at the fixed index KT-1.  A point enters iff its distance
// is strictly below the bound.
#pragma once

#include "bkd_internal.h"

namespace bkd {

__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// Sorted insertion of (dv, id) into an ascending list; requires dv < L[KT-1].
template <int KT>
__device__ __forceinline__ void list_insert(float (&Ld)[KT], uint32_t (&Li)[KT],
                                            float dv, uint32_t id) {
#pragma unroll
  for (int i = KT - 1; i > 0; --i) {
    const bool up = dv < Ld[i - 1];
    const bool here = dv < Ld[i];
    Li[i] = up ? Li[i - 1] : (here ? id : Li[i]);
    Ld[i] = up ? Ld[i - 1] : (here ? dv : Ld[i]);
  }
  if (dv < Ld[0]) {
    Ld[0] = dv;
    Li[0] = id;
  }
}

// Float32 distances of one query (coordinates duplicated into packed pairs
// qq[i] = (q_i, q_i)) to the four points of a quad b[0..D).
template <int D>
__device__ __forceinline__ void quad_dist(const float4* __restrict__ b,
                                          const uint64_t (&qq)[D], float& e0,
                                          float& e1, float& e2, float& e3) {
  uint64_t a01, a23;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const float4 v = b[i];
    const uint64_t d01 = sub2(qq[i], pk2(v.x, v.y));
    const uint64_t d23 = sub2(qq[i], pk2(v.z, v.w));
    if (i == 0) {
      a01 = mul2(d01, d01);
      a23 = mul2(d23, d23);
    } else {
      a01 = fma2(d01, d01, a01);
      a23 = fma2(d23, d23, a23);
    }
  }
  upk2(a01, e0, e1);
  upk2(a23, e2, e3);
}

// ---------------------------------------------------------------- TMA
// 1-D bulk copies (cp.async.bulk) global -> shared, completed on an mbarrier
// (transaction-count form).  Waits are bounded by the SM clock: a wait that
// runs out reports failure instead of spinning forever.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar),
               "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void async_proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Arms `bar` for `bytes` of transactions and starts one bulk copy into it.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src,
                                          uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::
                   "r"(bar),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(bar)
      : "memory");
}
// Waits for phase `parity` of `bar` to complete; false after ~2^31 cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

constexpr int kPipeThreads = 64;   // 2 warps: one query per thread
constexpr int kPipeSegQuads = 32;  // quads (128 points) per staged segment

// Producer side of the segment pipeline (thread 0 only): the (item, segment)
// sequence of this CTA, in the order the consumers walk it.
struct SegCursor {
  int it, seg, nseg;
};

// The quads [x, y) of a leaf of `cnt` points that a launch scans: all of
// them, or -- for the point-split chunks of Sec. 3.2 -- those holding the
// leaf-structure positions [part.pos_lo, part.pos_hi) (a multiple of 4
// points from the leaf's start, by construction of the chunk bounds).
__device__ __forceinline__ int2 quad_range(const LeafPart& part, int leaf,
                                           int cnt) {
  int lo = 0, hi = cnt;
  if (part.leaf_lo) {
    const int64_t b = part.leaf_lo[leaf];
    lo = (int)max((int64_t)0, part.pos_lo - b);
    hi = (int)min((int64_t)cnt, part.pos_hi - b);
  }
  return make_int2(lo >> 2, (hi + 3) >> 2);
}

__device__ __forceinline__ int segments_of(const Item* __restrict__ items,
                                           const int32_t* __restrict__ cnt,
                                           int it, const LeafPart& part) {
  const int leaf = items[it].leaf;
  const int2 r = quad_range(part, leaf, cnt[leaf]);
  return (r.y - r.x + kPipeSegQuads - 1) / kPipeSegQuads;
}

// Starts the copy of the segment under the cursor into `dst`, then advances.
template <int D>
__device__ __forceinline__ void issue_segment(
    SegCursor& c, int hi, int stride, const Item* __restrict__ items,
    const int32_t* __restrict__ cnt, const float4* __restrict__ pts,
    int64_t leaf0, int64_t qpl, const LeafPart& part, float4* dst,
    uint32_t bar) {
  if (c.it >= hi) return;
  const Item w = items[c.it];
  const int2 r = quad_range(part, w.leaf, cnt[w.leaf]);
  const int q0 = r.x + c.seg * kPipeSegQuads;
  const int sq = min(kPipeSegQuads, r.y - q0);
  const float4* src = pts + ((int64_t)(w.leaf - leaf0) * qpl + q0) * D;
  bulk_load(smem_u32(dst), src, (uint32_t)(sq * D * 16), bar);
  if (++c.seg == c.nseg) {
    c.it += stride;
    c.seg = 0;
    if (c.it < hi) c.nseg = segments_of(items, cnt, c.it, part);
  }
}

// ProcessAllBuffers, pipelined: one 64-thread CTA per item of <= 64 queries
// of one leaf (one query per thread); the leaf is streamed through two
// shared-memory segment buffers of 128 points
// that one thread fills with TMA bulk copies, one segment ahead of the
// consumers and across item boundaries.  Small CTAs and small buffers keep
// many items resident per SM, so a partly filled item idles few lanes and
// copy latency hides behind the other CTAs' arithmetic.
template <int D, int KT>
__global__ void __launch_bounds__(kPipeThreads)
    leaf_pipe_kernel(const Item* __restrict__ items, int item_lo,
                     int item_hi, Counters* ctr,
                     const float4* __restrict__ pts, int64_t leaf0,
                     const int32_t* __restrict__ leaf_cnt, int64_t lcap,
                     const uint32_t* __restrict__ act,
                     const float* __restrict__ qpad,
                     float* __restrict__ lst_d, uint32_t* __restrict__ lst_i,
                     int K, const int32_t* __restrict__ count_dev,
                     LeafPart part) {
  __shared__ __align__(128) float4 buf[2][kPipeSegQuads * D];
  __shared__ __align__(8) uint64_t full[2];
  const int hi = item_hi >= 0 ? item_hi
                              : (count_dev ? *count_dev : ctr->n_items);
  const int tid = threadIdx.x;
  const int64_t qpl = lcap >> 2;
  const int sent = KT - K;
  const uint32_t bar0 = smem_u32(&full[0]), bar1 = smem_u32(&full[1]);
  SegCursor cur{item_lo + (int)blockIdx.x, 0, 0};
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    mbar_init_fence();
    if (cur.it < hi) cur.nseg = segments_of(items, leaf_cnt, cur.it, part);
  }
  __syncthreads();
  if (tid == 0) {
    issue_segment<D>(cur, hi, gridDim.x, items, leaf_cnt, pts, leaf0, qpl,
                     part, buf[0], bar0);
    issue_segment<D>(cur, hi, gridDim.x, items, leaf_cnt, pts, leaf0, qpl,
                     part, buf[1], bar1);
  }
  uint32_t par0 = 0u, par1 = 0u;  // phase parity of each buffer's barrier
  int slot = 0;
  for (int it = item_lo + blockIdx.x; it < hi; it += gridDim.x) {
    const Item w = items[it];
    const int2 qr = quad_range(part, w.leaf, leaf_cnt[w.leaf]);
    const int nq = qr.y;
    const int nseg = (qr.y - qr.x + kPipeSegQuads - 1) / kPipeSegQuads;
    if (tid == 0) {
      atomicAdd(&ctr->leaf_pairs,
                (unsigned long long)w.count *
                    (unsigned long long)min(leaf_cnt[w.leaf] - 4 * qr.x,
                                            4 * (qr.y - qr.x)));
      atomicAdd(&ctr->leaf_bytes,
                (unsigned long long)(qr.y - qr.x) * (16u * D));
    }
    const bool on = tid < w.count;
    uint32_t q = 0;
    uint64_t qq[D];
    float Ld[KT];
    uint32_t Li[KT];
    if (on) {
      q = act[w.start + tid];
      const float* qp = qpad + (size_t)q * D;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const float x = qp[i];
        qq[i] = pk2(x, x);
      }
#pragma unroll
      for (int i = 0; i < KT; ++i) {
        if (i < sent) {
          Ld[i] = -1.f;
          Li[i] = kNoSlot;
        } else {
          Ld[i] = lst_d[(size_t)q * K + (i - sent)];
          Li[i] = lst_i[(size_t)q * K + (i - sent)];
        }
      }
    }
    const uint32_t slot0 = (uint32_t)((int64_t)w.leaf * lcap);
    for (int sg = 0; sg < nseg; ++sg) {
      const bool ok = mbar_wait(slot ? bar1 : bar0, slot ? par1 : par0);
      if (__syncthreads_or(!ok)) {
        // a copy never completed: report, give the copies in flight a
        // bounded chance to land, and leave without touching the buffers
        if (tid == 0) {
          atomicOr(&ctr->err, kErrTimeout);
          mbar_wait(bar0, par0);
          mbar_wait(bar1, par1);
        }
        return;
      }
      if (slot)
        par1 ^= 1u;
      else
        par0 ^= 1u;
      if (on) {
        const float4* b = buf[slot];
        const int q0 = qr.x + sg * kPipeSegQuads;
        const int sq = min(kPipeSegQuads, nq - q0);
        float bound = Ld[KT - 1];
#pragma unroll 2
        for (int g = 0; g < sq; ++g) {
          float e0, e1, e2, e3;
          quad_dist<D>(b + g * D, qq, e0, e1, e2, e3);
          if (fminf(fminf(e0, e1), fminf(e2, e3)) < bound) {
            const uint32_t id = slot0 + (uint32_t)(q0 + g) * 4u;
            if (e0 < bound) {
              list_insert<KT>(Ld, Li, e0, id);
              bound = Ld[KT - 1];
            }
            if (e1 < bound) {
              list_insert<KT>(Ld, Li, e1, id + 1);
              bound = Ld[KT - 1];
            }
            if (e2 < bound) {
              list_insert<KT>(Ld, Li, e2, id + 2);
              bound = Ld[KT - 1];
            }
            if (e3 < bound) {
              list_insert<KT>(Ld, Li, e3, id + 3);
              bound = Ld[KT - 1];
            }
          }
        }
      }
      __syncthreads();  // both warps are done with buf[slot]
      if (tid == 0) {
        async_proxy_fence();
        issue_segment<D>(cur, hi, gridDim.x, items, leaf_cnt, pts, leaf0, qpl,
                         part, buf[slot], slot ? bar1 : bar0);
      }
      slot ^= 1;
    }
    if (on) {
#pragma unroll
      for (int i = 0; i < KT; ++i) {
        if (i >= sent) {
          lst_d[(size_t)q * K + (i - sent)] = Ld[i];
          lst_i[(size_t)q * K + (i - sent)] = Li[i];
        }
      }
    }
  }
}

// Per-capacity launchers, defined once per capacity in k_leaf_c<KT>.cu.
#define BKD_LEAF_ARGS                                                        \
  int Dp, const Item *items, int item_lo, int item_hi, Counters *ctr,       \
      const float *pts, int64_t leaf0, const int32_t *leaf_cnt,             \
      int64_t lcap, const uint32_t *act, const float *qpad, float *lst_d,   \
      uint32_t *lst_i, int K, int grid, cudaStream_t s,                     \
      const int32_t *count_dev, LeafPart part

#define BKD_LEAF_DECLARE(CAP)                    \
  cudaError_t leaf_launch_c##CAP(BKD_LEAF_ARGS); \
  const void* leaf_kernel_c##CAP(int Dp);

BKD_LEAF_DECLARE(2)
BKD_LEAF_DECLARE(4)
BKD_LEAF_DECLARE(8)
BKD_LEAF_DECLARE(12)
BKD_LEAF_DECLARE(16)
BKD_LEAF_DECLARE(32)
BKD_LEAF_DECLARE(64)

#define BKD_LEAF_DIMS(X) BKD_DIMS(X)

#define BKD_LEAF_CASE_LAUNCH(DIM)                                             \
  case DIM:                                                                   \
    leaf_pipe_kernel<DIM, KT><<<grid, kPipeThreads, 0, s>>>(                  \
        items, item_lo, item_hi, ctr, reinterpret_cast<const float4*>(pts),    \
        leaf0, leaf_cnt, lcap, act, qpad, lst_d, lst_i, K, count_dev, part);  \
    return cudaGetLastError();

#define BKD_LEAF_CASE_PTR(DIM) \
  case DIM:                    \
    return reinterpret_cast<const void*>(&leaf_pipe_kernel<DIM, KT>);

#define BKD_LEAF_DEFINE(CAP)                                            \
  cudaError_t leaf_launch_c##CAP(BKD_LEAF_ARGS) {                       \
    constexpr int KT = CAP;                                             \
    switch (Dp) { BKD_LEAF_DIMS(BKD_LEAF_CASE_LAUNCH) default: break; } \
    return cudaErrorInvalidValue;                                       \
  }                                                                     \
  const void* leaf_kernel_c##CAP(int Dp) {                              \
    constexpr int KT = CAP;                                             \
    switch (Dp) { BKD_LEAF_DIMS(BKD_LEAF_CASE_PTR) default: break; }    \
    return nullptr;                                                     \
  }

}  // namespace bkd
