// k_leaf.cuh -- ProcessAllBuffers: leaf brute force with the k-best merge
// fused in (Algorithm 1; Sec. 3.2 "each thread compares a particular query
// with all reference points stored in the associated leaf").
//
// One CTA takes one work item at a time: up to kTileQ buffered queries of one
// leaf.  The leaf's quads are staged in shared memory (segments of at most
// `seg_quads` quads); every thread owns one query, holds its coordinates and
// its sorted candidate list in registers and streams over the staged points,
// reading each quad with warp-broadcast float4 loads.
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

template <int D, int KT>
__global__ void __launch_bounds__(kTileQ)
    leaf_kernel(const Item* __restrict__ items, int item_lo, int item_hi,
                const Counters* __restrict__ ctr,
                const float4* __restrict__ pts, int64_t leaf0,
                const int32_t* __restrict__ leaf_cnt, int64_t lcap,
                const uint32_t* __restrict__ act,
                const float* __restrict__ qpad, float* __restrict__ lst_d,
                uint32_t* __restrict__ lst_i, int K, int seg_quads) {
  extern __shared__ float4 sm[];
  const int hi = item_hi >= 0 ? item_hi : ctr->n_items;
  const int tid = threadIdx.x;
  const int64_t qpl = lcap >> 2;  // quads per leaf
  const int sent = KT - K;        // sentinel entries in front of the list
  for (int it = item_lo + blockIdx.x; it < hi; it += gridDim.x) {
    const Item w = items[it];
    const int nq = (leaf_cnt[w.leaf] + 3) >> 2;
    const float4* src = pts + (int64_t)(w.leaf - leaf0) * qpl * D;
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
    for (int s0 = 0; s0 < nq; s0 += seg_quads) {
      const int sq = min(seg_quads, nq - s0);
      __syncthreads();  // the previous segment / item is no longer read
      const float4* seg = src + (int64_t)s0 * D;
      for (int i = tid; i < sq * D; i += kTileQ) sm[i] = seg[i];
      __syncthreads();
      if (on) {
        float bound = Ld[KT - 1];
#pragma unroll 2
        for (int g = 0; g < sq; ++g) {
          float e0, e1, e2, e3;
          quad_dist<D>(sm + g * D, qq, e0, e1, e2, e3);
          if (fminf(fminf(e0, e1), fminf(e2, e3)) < bound) {
            const uint32_t id = slot0 + (uint32_t)(s0 + g) * 4u;
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
#define BKD_LEAF_ARGS                                                       \
  int Dp, const Item *items, int item_lo, int item_hi, const Counters *ctr, \
      const float *pts, int64_t leaf0, const int32_t *leaf_cnt,             \
      int64_t lcap, const uint32_t *act, const float *qpad, float *lst_d,   \
      uint32_t *lst_i, int K, int grid, int seg_quads, size_t smem,         \
      cudaStream_t s

#define BKD_LEAF_DECLARE(CAP)                           \
  cudaError_t leaf_launch_c##CAP(BKD_LEAF_ARGS);        \
  const void* leaf_kernel_c##CAP(int Dp);

BKD_LEAF_DECLARE(2)
BKD_LEAF_DECLARE(4)
BKD_LEAF_DECLARE(8)
BKD_LEAF_DECLARE(12)
BKD_LEAF_DECLARE(16)
BKD_LEAF_DECLARE(32)

#define BKD_LEAF_DIMS(X) X(2) X(4) X(6) X(8) X(10) X(12) X(16) X(24) X(32)

#define BKD_LEAF_CASE_LAUNCH(DIM)                                          \
  case DIM:                                                                \
    leaf_kernel<DIM, KT><<<grid, kTileQ, smem, s>>>(                       \
        items, item_lo, item_hi, ctr, reinterpret_cast<const float4*>(pts), \
        leaf0, leaf_cnt, lcap, act, qpad, lst_d, lst_i, K, seg_quads);     \
    return cudaGetLastError();

#define BKD_LEAF_CASE_PTR(DIM) \
  case DIM:                    \
    return reinterpret_cast<const void*>(&leaf_kernel<DIM, KT>);

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
