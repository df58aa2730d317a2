// k_exact.cu -- turning the float32 candidate lists into exact answers.
//
// After LazySearch every query holds the k+1 smallest float32 distances
// v_0 <= ... <= v_k over all n points (exact pruning, see k_traverse.cu).
// The answer is defined by binary64 distances and the smaller-index tie rule
// (Sec. 2.2 problem statement).  With u = 2^-24 the float32 value of a
// distance D64 obeys |v - D64| <= gam * D64 + eta, gam = (d + 3) u (the
// d+2 roundings of the float32 chain plus the binary64 rounding of D64, with
// margin) and eta = 2^-120 (subnormal underflow).  Hence D64 lies in
// [lo(v), hi(v)] with lo(v) = (v - eta) / (1 + gam), hi(v) = (v + eta) /
// (1 - gam), and "a certainly below b" means hi(a) < lo(b).
//
//   * k-th certainly below (k+1)-th: the first k list entries are exactly
//     the k nearest points (every other point scores >= v_k).
//       - all adjacent entries certainly ordered: the float32 order is the
//         exact order; output as is.
//       - otherwise: recompute the k distances in binary64 (same operation
//         order as the oracle) and sort by (D64, index).
//   * otherwise (a near tie at the k / k+1 boundary): the query is searched
//     again in binary64 by the fallback kernel below, a classical depth-first
//     k-d tree search (Sec. 2.3) with the exact key, skipping subtrees whose
//     binary64 bounding-box distance exceeds min(current k-th D64,
//     hi(v_{k-1})) -- hi(v_{k-1}) bounds the true k-th distance from above
//     because k points score at most v_{k-1}.  The traversal and the point
//     filter compare float32 values against that bound widened to
//     r (1 + gam) + eta (every point or box with D64 <= r scores at most
//     that in float32); a point's binary64 distance is formed only when it
//     passes.
#include <cmath>

#include "bkd.h"
#include "bkd_internal.h"
#include "traverse.cuh"

namespace bkd {
namespace {

// The interval [lo(v), hi(v)] with directed roundings: `rlo` <= 1/(1+gam)
// and `rhi` >= 1/(1-gam) are prepared on the host (Bounds), so the interval
// only widens.
struct Bounds {
  double eta, rlo, rhi;
  double gup;  // >= 1 + gam
};
__device__ __forceinline__ double lo_bound(float v, const Bounds& b) {
  return __dmul_rd(__dsub_rd((double)v, b.eta), b.rlo);
}
__device__ __forceinline__ double hi_bound(float v, const Bounds& b) {
  return __dmul_ru(__dadd_ru((double)v, b.eta), b.rhi);
}

__device__ __forceinline__ float coord(const float* pts, int Dp, uint64_t slot,
                                       int i) {
  return pts[(slot >> 2) * 4 * (uint64_t)Dp + 4 * i + (slot & 3)];
}

// binary64 squared distance, terms added in dimension order from 0.0 with
// one rounding per operation (the oracle's sequence).
__device__ double dist64(const float* qp, const float* pts, int Dp, int d,
                         uint64_t slot) {
  double acc = 0.0;
  for (int i = 0; i < d; ++i) {
    const double t = __dsub_rn((double)qp[i], (double)coord(pts, Dp, slot, i));
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

// float32 squared distance by the leaf kernel's chain (the value v above):
// e = fl(t_0^2), e = fma(t_i, t_i, e), t_i = fl(q_i - x_i).
__device__ float dist32(const float* qp, const float* pts, int Dp, int d,
                        uint64_t slot) {
  float t = __fsub_rn(qp[0], coord(pts, Dp, slot, 0));
  float e = __fmul_rn(t, t);
  for (int i = 1; i < d; ++i) {
    t = __fsub_rn(qp[i], coord(pts, Dp, slot, i));
    e = __fmaf_rn(t, t, e);
  }
  return e;
}

__device__ __forceinline__ bool key_less(double da, int64_t ia, double db,
                                         int64_t ib) {
  return da < db || (da == db && ia < ib);
}

__global__ void recheck_kernel(DevTree t, int64_t m, int k, int K,
                               const float* __restrict__ qpad,
                               const float* __restrict__ lst_d,
                               const uint32_t* __restrict__ lst_i,
                               int64_t* __restrict__ out_idx,
                               float* __restrict__ out_dist,
                               uint32_t* __restrict__ fb_list, Counters* ctr,
                               Bounds bd) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  const float* v = lst_d + q * K;
  const uint32_t* sl = lst_i + q * K;
  // Every finished list holds k real entries (k <= n and finite inputs make
  // every point score finitely); anything else is reported, never followed.
  const uint64_t nslots = (uint64_t)t.lcap << t.h;
  for (int j = 0; j < k; ++j) {
    if ((uint64_t)sl[j] >= nslots) {
      atomicOr(&ctr->err, kErrBadList);
      for (int i = 0; i < k; ++i) {
        out_idx[q * k + i] = -1;
        out_dist[q * k + i] = __int_as_float(0x7fc00000);
      }
      return;
    }
  }
  const float vk = v[k];
  const bool member_ok =
      isinf(vk) || hi_bound(v[k - 1], bd) < lo_bound(vk, bd);
  if (!member_ok) {
    const int j = atomicAdd(&ctr->n_fallback, 1);
    fb_list[j] = (uint32_t)q;
    return;
  }
  bool order_ok = true;
  for (int j = 0; j + 1 < k; ++j)
    order_ok &= hi_bound(v[j], bd) < lo_bound(v[j + 1], bd);
  if (order_ok) {
    for (int j = 0; j < k; ++j) {
      out_idx[q * k + j] = t.orig[sl[j]];
      out_dist[q * k + j] = v[j];
    }
    return;
  }
  atomicAdd(&ctr->n_resorted, 1);
  double dd[BKD_MAX_K];
  int64_t ii[BKD_MAX_K];
  const float* qp = qpad + q * t.Dp;
  for (int j = 0; j < k; ++j) {
    const double dv = dist64(qp, t.pts, t.Dp, t.d, sl[j]);
    const int64_t iv = t.orig[sl[j]];
    int p = j;
    while (p > 0 && key_less(dv, iv, dd[p - 1], ii[p - 1])) {
      dd[p] = dd[p - 1];
      ii[p] = ii[p - 1];
      --p;
    }
    dd[p] = dv;
    ii[p] = iv;
  }
  for (int j = 0; j < k; ++j) {
    out_idx[q * k + j] = ii[j];
    out_dist[q * k + j] = (float)dd[j];
  }
}

// A binary64 distance bound r as a float32 bound on the float32 chain: a
// point or box with D64 <= r scores v <= r (1 + gam) + eta, rounded up here;
// returned as the next float above it, for the strict test of F32Bound.
__device__ __forceinline__ float f32_bound(double r, const Bounds& b) {
  if (isinf(r)) return __int_as_float(0x7f800000);
  const float v = __double2float_ru(__dadd_ru(__dmul_ru(r, b.gup), b.eta));
  if (isinf(v)) return v;
  return __int_as_float(__float_as_int(v) + 1);  // v >= 0: the next float
}

// One warp per query (one warp per CTA, so that the few fallback queries
// spread over the SMs).  The sorted binary64 list (k entries) lives in
// shared memory; candidates -- rare: only points that pass the float32
// filter -- are inserted by lane 0 one at a time.  The traversal and the
// point filter run on float32 values with the bound widened by f32_bound
// (the binary64 pipe is narrow); only points that pass get their binary64
// distance.
template <int D>
__global__ void __launch_bounds__(32)
    fallback_kernel(DevTree t, int n_fb, const uint32_t* __restrict__ fb_list,
                    int k, int K, const float* __restrict__ qpad,
                    const float* __restrict__ lst_d,
                    int64_t* __restrict__ out_idx,
                    float* __restrict__ out_dist, Bounds bd, Counters* ctr) {
  __shared__ double s_d[BKD_MAX_K];
  __shared__ int64_t s_i[BKD_MAX_K];
  const int lane = threadIdx.x & 31;
  const int first_leaf = (1 << t.h) - 1;
  for (int f = blockIdx.x; f < n_fb; f += gridDim.x) {
    const int64_t q = fb_list[f];
    const float* qp = qpad + q * D;
    F32Bound<D> bx;
    bx.load(qp);
    const double seed = hi_bound(lst_d[q * K + (k - 1)], bd);
    const float seed32 = f32_bound(seed, bd);
    int cnt = 0;  // entries in the list (warp-uniform)
    unsigned long long scanned = 0;  // points of the leaves scanned (lane 0)
    int node = kStart;
    uint32_t mask = 0;
    for (;;) {
      // the bound: min(k-th D64, seed) once the list is full
      const double r = cnt == k ? fmin(s_d[k - 1], seed) : seed;
      node = next_leaf(t, bx, qp, node, mask, f32_bound(r, bd));
      if (node == kDone) break;
      // ---- scan the leaf
      const int leaf = node - first_leaf;
      const int np = t.leaf_cnt[leaf];
      const uint64_t base = (uint64_t)leaf * (uint64_t)t.lcap;
      if (lane == 0) scanned += (unsigned long long)np;
      for (int u0 = 0; u0 < np; u0 += 32) {
        const int u = u0 + lane;
        double dv = 0.0;
        int64_t iv = 0;
        bool cand = false;
        if (u < np && dist32(qp, t.pts, D, t.d, base + u) < seed32) {
          dv = dist64(qp, t.pts, D, t.d, base + u);
          iv = t.orig[base + u];
          cand = dv <= seed;
        }
        unsigned m = __ballot_sync(0xffffffffu, cand);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          const double cd = __shfl_sync(0xffffffffu, dv, src);
          const int64_t ci = __shfl_sync(0xffffffffu, iv, src);
          if (lane == 0 &&
              (cnt < k || key_less(cd, ci, s_d[k - 1], s_i[k - 1]))) {
            int p = cnt < k ? cnt : k - 1;
            while (p > 0 && key_less(cd, ci, s_d[p - 1], s_i[p - 1])) {
              s_d[p] = s_d[p - 1];
              s_i[p] = s_i[p - 1];
              --p;
            }
            s_d[p] = cd;
            s_i[p] = ci;
          }
          cnt = min(cnt + 1, k);
          __syncwarp();
        }
      }
    }
    for (int j = lane; j < k; j += 32) {
      out_idx[q * k + j] = s_i[j];
      out_dist[q * k + j] = (float)s_d[j];
    }
    if (ctr && lane == 0 && scanned) atomicAdd(&ctr->fallback_points, scanned);
    __syncwarp();
  }
}

// gam = (d + 3) 2^-24, eta = 2^-120; the reciprocals rounded outward.
Bounds bounds_for(int d) {
  const double gam = (d + 3) * 5.9604644775390625e-08;
  Bounds b;
  b.eta = 7.52316384526264e-37;
  b.rlo = std::nextafter(1.0 / (1.0 + gam), 0.0);
  b.rhi = std::nextafter(1.0 / (1.0 - gam), 2.0);
  b.gup = std::nextafter(1.0 + gam, 2.0);
  return b;
}

}  // namespace

cudaError_t launch_recheck(const DevTree& t, int64_t m, int k, int K,
                           const float* qpad, const float* lst_d,
                           const uint32_t* lst_i, int64_t* out_idx,
                           float* out_dist, uint32_t* fb_list, Counters* ctr,
                           cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  recheck_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(
      t, m, k, K, qpad, lst_d, lst_i, out_idx, out_dist, fb_list, ctr,
      bounds_for(t.d));
  return cudaGetLastError();
}

cudaError_t launch_fallback(const DevTree& t, int n_fb, const uint32_t* fb_list,
                            int k, int K, const float* qpad, const float* lst_d,
                            int64_t* out_idx, float* out_dist, cudaStream_t s,
                            Counters* ctr) {
  if (n_fb == 0) return cudaSuccess;
  const int grid = n_fb < 65536 ? n_fb : 65536;
#define BKD_FB_CASE(DIM)                                                  \
  case DIM:                                                               \
    fallback_kernel<DIM><<<grid, 32, 0, s>>>(t, n_fb, fb_list, k, K, qpad, \
                                             lst_d, out_idx, out_dist,     \
                                             bounds_for(t.d), ctr);        \
    return cudaGetLastError();
  switch (t.Dp) { BKD_DIMS(BKD_FB_CASE) default: break; }
#undef BKD_FB_CASE
  return cudaErrorInvalidValue;
}

}  // namespace bkd
