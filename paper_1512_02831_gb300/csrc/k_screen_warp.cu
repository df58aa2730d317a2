// k_screen_warp.cu -- ProcessAllBuffers with a BF16 tensor-core screen,
// one warp per work item (mma.sync; the default screen kernel).
//
// Same candidate lists as the float32 leaf kernel (every point whose float32
// distance could still enter a query's list is scored exactly), but most
// points are rejected by a cheap screen first:
//
//   v = q - c, w = x - c (c: centre of the leaf), rounded to bf16 (v^, w^);
//   s = |v^|^2 + |w^|^2 - 2 v^.w^.
//
// The tensor cores form D = v^.w^ - |w^|^2/2 (mma.sync m16n8k16, bf16 in,
// fp32 accumulate from zero): 16 points (rows) x 8 queries (columns) per
// instruction and k-half of 16 bf16 slots.  A point's slots hold w^ and,
// after it, pn_hi and pn_lo (pn = fl32(|w^|^2), pn_hi = bf16(pn), pn_lo =
// bf16(pn - pn_hi), so |w^|^2 = pn_hi + pn_lo up to (2^-16 + 2^-24) pn); a
// query's hold v^ and -1/2, -1/2.  So s = |v^|^2 - 2 D, and the screen test
// s < T reads D > (|v^|^2 - T) / 2: one comparison per (query, point) pair.
// Padding points carry pn_hi = +inf, so D = -inf there.
//
// Safety bound.  bf16 keeps 8 significant bits, so round-to-nearest errs by
// at most 2^-8 relative; with the float32 subtraction before it, rho =
// 2^-8 (1 + 1e-4) and |v^ - v| <= rho |v|, |v| <= |v^| / (1 - rho), so
//   |q - x| >= |v^ - w^| - A_q - B_x,  A_q = rho/(1-rho) |v^|,
// and B_x <= B_max, the leaf's largest such term (prepared on the host).
// The computed s differs from |v^ - w^|^2 by at most
//   E = 2^-14 (|v^|^2 + pn_max):
//   * accumulation model: one MMA (16 exact bf16 products added to an fp32
//     accumulator c) errs by at most 2^-18 (|c| + sum |a_i b_i|); the KH
//     chained halves of one pair then err by at most KH 2^-18 S, S = the sum
//     of the absolute products <= |v^|^2 / 2 + pn (1 + 2^-8).  (A hardware
//     property, not an IEEE rule: the bf16 MMA probe test checks it on
//     adversarial operands -- one large term and many small ones,
//     cancellation, mixed exponents within a k-half.)  With KH <= 3 the
//     error of s = |v^|^2 - 2D is <= 2^-16.4 |v^|^2 + 2^-15.4 pn;
//   * the norm split adds (2^-16 + 2^-24) pn, the float32 chain of |v^|^2
//     at most d 2^-24 |v^|^2 <= 2^-19 |v^|^2;
//   * in total < 1.4e-5 |v^|^2 + 3.9e-5 pn <= E (2^-14 = 6.1e-5).
// The float32 distance of the exact path obeys D32 >= D (1 - g) - eta,
// g = (d+3) 2^-24, eta = 2^-120.  Hence a point can only enter the list
// (D32 < bound) if
//   s < T = (sqrt((bound + eta) / (1 - g)) + A_q + B_max)^2 + E,
// evaluated once per (query, leaf) in float32 with every operation rounded
// toward the larger threshold (divisors toward the smaller).  Kept points
// are scored with the exact float32 chain of the leaf kernel and inserted
// with the same strict rule in ascending slot order, so the lists -- and the
// answers -- are bit for bit those of the float32 path.
//
// Work layout.  One warp per item (one leaf, at most 32 buffered queries,
// i.e. up to four 8-query column blocks).  Each lane streams its own A
// fragments of the leaf through a small shared-memory ring (cp.async, L2
// only).  Kept pairs go to a per-warp queue; a full queue is scored 32
// pairs at a time and inserted per query in queue order.  A query's list is
// read from global memory only when a point is inserted into it, and
// written back only then.
#include <cuda_bf16.h>

#include <algorithm>

#include "bkd.h"
#include "bkd_internal.h"

namespace bkd {
namespace {

constexpr int kScrWarps = 8;
constexpr int kScrThreads = kScrWarps * 32;
constexpr int kQueue = 64;  // kept pairs per warp between two scorings
static_assert(kWarpScreenTile == 32, "one query column per lane");

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float bf16_lo(uint32_t w) {
  return __uint_as_float(w << 16);
}
__device__ __forceinline__ float bf16_hi(uint32_t w) {
  return __uint_as_float(w & 0xffff0000u);
}

// acc = a (16x16 bf16, row) x b (16x8 bf16, col) + acc, fp32.
__device__ __forceinline__ void mma_bf16(float (&acc)[4], uint32_t a0,
                                         uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// acc = a x b, accumulated from zero.
__device__ __forceinline__ void mma_bf16_z(float (&acc)[4], uint32_t a0,
                                           uint32_t a1, uint32_t a2,
                                           uint32_t a3, uint32_t b0,
                                           uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%10, %10, %10, %10};"
      : "=f"(acc[0]), "=f"(acc[1]), "=f"(acc[2]), "=f"(acc[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(0.f));
}

// max(a, b, c) (three-input float max of sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Exact float32 distance of query coordinates qp (Dp, zero-padded) to the
// point in `slot`: the leaf kernel's chain, one dimension at a time.
__device__ __forceinline__ float exact_dist(const float* __restrict__ qp,
                                            const float* __restrict__ pts,
                                            int Dp, uint32_t slot) {
  const float* quad = pts + (size_t)(slot >> 2) * 4 * Dp + (slot & 3);
  float t = __fsub_rn(qp[0], quad[0]);
  float e = __fmul_rn(t, t);
  for (int i = 1; i < Dp; ++i) {
    t = __fsub_rn(qp[i], quad[4 * i]);
    e = __fmaf_rn(t, t, e);
  }
  return e;
}

// Per-warp shared memory (32-bit words):
//   ring   R x NC x 32 x 4  super-tiles in flight: stage, component, lane
//                       (each lane copies, and later reads, only its own
//                       fragments; NC = 2 KH 16-byte components)
//   rec    32 x KH x 8   bf16 offsets of the item's queries (B operand)
//   tneg   32            -T'/2 per query column (+inf: unused column)
//   qid    32            query ids
//   bound  32            last entry of each column's candidate list
//   flag   32            bit 0: list copied into ld/li, bit 1: list changed
//   queue  kQueue        kept pairs: (slot in leaf) << 5 | column
//   qd     kQueue        their exact float32 distances
//   ld, li 32 x K each   candidate lists, read on first insertion
struct WarpSmem {
  uint4* ring;
  uint32_t* rec;
  float* tneg;
  uint32_t* qid;
  float* bound;
  uint32_t* flag;
  uint32_t* queue;
  float* qd;
  float* ld;
  uint32_t* li;
};

// Ring depth (super-tiles per warp in the ring: one being read, the rest in
// flight) and 16-byte components per stage.  Measured best at 3 (with three
// CTAs per SM); deeper rings are slower: their shared memory comes out of
// L1.
__host__ __device__ constexpr int ring_depth(int) { return 3; }
__host__ __device__ constexpr int ring_comps(int kh) { return 2 * kh; }

__host__ __device__ constexpr int warp_words(int kh, int K) {
  return ring_depth(kh) * ring_comps(kh) * 128 + kh * 256 + 128 +
         2 * kQueue + 64 * K;
}

template <int KH>
__device__ __forceinline__ WarpSmem warp_smem(uint32_t* base, int warp,
                                              int K) {
  uint32_t* p = base + (size_t)warp * warp_words(KH, K);
  WarpSmem w;
  w.ring = reinterpret_cast<uint4*>(p);
  p += ring_depth(KH) * ring_comps(KH) * 128;
  w.rec = p;
  w.tneg = reinterpret_cast<float*>(p + KH * 256);
  w.qid = p + KH * 256 + 32;
  w.bound = reinterpret_cast<float*>(w.qid + 32);
  w.flag = w.qid + 64;
  w.queue = w.qid + 96;
  w.qd = reinterpret_cast<float*>(w.queue + kQueue);
  w.ld = w.qd + kQueue;
  w.li = reinterpret_cast<uint32_t*>(w.ld + 32 * K);
  return w;
}

// Scores the queued pairs (one per lane at a time) and inserts them, per
// query column, in queue order -- which is ascending slot order per column.
// Out of line: it runs for a few tiles only, and inlined copies would crowd
// the instruction cache.
__device__ __noinline__ void drain(const DevTree& t, int leaf,
                                   const float* __restrict__ qpad,
                                   const float* __restrict__ lst_d,
                                   const uint32_t* __restrict__ lst_i, int K,
                                   const WarpSmem& ws, int lane, int nq,
                                   int ncol, uint32_t pofs) {
  __syncwarp();
  const uint32_t slot0 = (uint32_t)((int64_t)leaf * t.lcap);
  for (int e = lane; e < nq; e += 32) {
    const uint32_t en = ws.queue[e];
    const uint32_t q = ws.qid[en & 31u];
    // (t.pts from slot pofs on: a chunk buffer on chunked trees)
    ws.qd[e] = exact_dist(qpad + (size_t)q * t.Dp, t.pts, t.Dp,
                          slot0 + (en >> 5) - pofs);
  }
  __syncwarp();
  if (lane < ncol) {
    float* ld = ws.ld + lane * K;
    uint32_t* li = ws.li + lane * K;
    const uint32_t q = ws.qid[lane];
    float bound = ws.bound[lane];
    uint32_t flag = ws.flag[lane];
    for (int e = 0; e < nq; ++e) {
      const uint32_t en = ws.queue[e];
      if ((int)(en & 31u) != lane) continue;
      const float dv = ws.qd[e];
      if (!(dv < bound)) continue;
      if (!(flag & 1u)) {
        for (int j = 0; j < K; ++j) {
          ld[j] = lst_d[(size_t)q * K + j];
          li[j] = lst_i[(size_t)q * K + j];
        }
      }
      int pos = K - 1;
      while (pos > 0 && ld[pos - 1] > dv) {
        ld[pos] = ld[pos - 1];
        li[pos] = li[pos - 1];
        --pos;
      }
      ld[pos] = dv;
      li[pos] = slot0 + (en >> 5);
      bound = ld[K - 1];
      flag = 3u;
    }
    ws.bound[lane] = bound;
    ws.flag[lane] = flag;
  }
  __syncwarp();
}

// One 32-point super-tile in registers: per k-half the A fragments of rows
// g and g + 8 of both m-tiles.
template <int KH>
struct Super {
  uint4 a[KH][2];
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copies this lane's fragments of super-tile S into ring stage `slot`.
template <int KH>
__device__ __forceinline__ void issue_super(const WarpSmem& ws, int slot,
                                            int lane, const uint4* wb,
                                            int64_t hstep, int S) {
  uint4* dst = ws.ring + (size_t)slot * ring_comps(KH) * 32 + lane;
  const uint4* src = wb + (int64_t)S * 64;
#pragma unroll
  for (int h = 0; h < KH; ++h) {
    cp_async16(dst + (2 * h) * 32, src + h * hstep);
    cp_async16(dst + (2 * h + 1) * 32, src + h * hstep + 32);
  }
}

template <int KH>
__device__ __forceinline__ void read_super(Super<KH>& x, const WarpSmem& ws,
                                           int slot, int lane) {
  const uint4* src = ws.ring + (size_t)slot * ring_comps(KH) * 32 + lane;
#pragma unroll
  for (int h = 0; h < KH; ++h) {
    x.a[h][0] = src[(2 * h) * 32];
    x.a[h][1] = src[(2 * h + 1) * 32];
  }
}

// acc[nb] = (m-tile a of x) . (column block nb of b) = v^.w^ - |w^|^2 / 2.
template <int KH, int NB>
__device__ __forceinline__ void super_mma(float (&acc)[NB][4],
                                          const Super<KH>& x,
                                          const uint32_t (&b)[NB][KH][2],
                                          int a) {
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
#pragma unroll
    for (int h = 0; h < KH; ++h) {
      const uint4 r0 = x.a[h][0], r1 = x.a[h][1];
      const uint32_t a0 = a ? r0.z : r0.x, a1 = a ? r1.z : r1.x,
                     a2 = a ? r0.w : r0.y, a3 = a ? r1.w : r1.y;
      if (h == 0)
        mma_bf16_z(acc[nb], a0, a1, a2, a3, b[nb][h][0], b[nb][h][1]);
      else
        mma_bf16(acc[nb], a0, a1, a2, a3, b[nb][h][0], b[nb][h][1]);
    }
  }
}

// The screen over one leaf for NB 8-query column blocks, one 32-point
// super-tile (two m16n8k16 m-tiles) per step, with ring_depth - 1 further
// super-tiles on their way into shared memory (cp.async).
template <int KH, int NB>
__device__ __forceinline__ void scan_leaf(
    const DevTree& t, const ScreenData& sc, int leaf, int npt,
    const WarpSmem& ws, int lane, const float* __restrict__ qpad,
    const float* __restrict__ lst_d, const uint32_t* __restrict__ lst_i,
    int K, int ncol, unsigned long long& kept) {
  const int g = lane >> 2, tq = lane & 3;
  const unsigned full = 0xffffffffu;
  uint32_t b[NB][KH][2];
  float tn[NB][2];
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
#pragma unroll
    for (int h = 0; h < KH; ++h) {
      const uint2 v = *reinterpret_cast<const uint2*>(
          ws.rec + ((nb * 8 + g) * KH + h) * 8 + 2 * tq);
      b[nb][h][0] = v.x;
      b[nb][h][1] = v.y;
    }
    tn[nb][0] = ws.tneg[nb * 8 + 2 * tq];
    tn[nb][1] = ws.tneg[nb * 8 + 2 * tq + 1];
  }
  const int64_t st = sc.stride;
  const int64_t hstep = st * 2;  // uint4 per k-half of a leaf
  const uint4* wb = reinterpret_cast<const uint4*>(sc.wwords) +
                    (size_t)(leaf - sc.leaf0) * KH * hstep + g * 4 + tq;
  const int nsup = (npt + 31) >> 5;
  constexpr int R = ring_depth(KH);
#pragma unroll
  for (int j = 0; j < R - 1; ++j) {
    if (j < nsup) issue_super<KH>(ws, j, lane, wb, hstep, j);
    cp_async_commit();  // possibly empty: one group per super-tile
  }
  int nq = 0;
  int slot = 0, fill = R - 1;  // stage read now, stage refilled now
  for (int S = 0; S < nsup; ++S) {
    // the stage refilled was read in the previous step (its values were
    // consumed by the multiplications there)
    if (S + R - 1 < nsup) issue_super<KH>(ws, fill, lane, wb, hstep, S + R - 1);
    cp_async_commit();
    cp_async_wait<R - 1>();  // super-tile S has landed
    Super<KH> x;
    read_super<KH>(x, ws, slot, lane);
    slot = slot + 1 == R ? 0 : slot + 1;
    fill = fill + 1 == R ? 0 : fill + 1;
    // the hot path only asks whether any pair of the super-tile passes:
    // per query column the largest D over its 4 rows (2 per m-tile)
    float cm[NB][2];
    {
      float acc[NB][4];
      super_mma<KH, NB>(acc, x, b, 0);
#pragma unroll
      for (int nb = 0; nb < NB; ++nb) {
        cm[nb][0] = fmaxf(acc[nb][0], acc[nb][2]);
        cm[nb][1] = fmaxf(acc[nb][1], acc[nb][3]);
      }
      super_mma<KH, NB>(acc, x, b, 1);
#pragma unroll
      for (int nb = 0; nb < NB; ++nb) {
        cm[nb][0] = fmax3(cm[nb][0], acc[nb][0], acc[nb][2]);
        cm[nb][1] = fmax3(cm[nb][1], acc[nb][1], acc[nb][3]);
      }
    }
    bool any = false;
#pragma unroll
    for (int nb = 0; nb < NB; ++nb)
      any = any || cm[nb][0] > tn[nb][0] || cm[nb][1] > tn[nb][1];
    if (__any_sync(full, any)) {
      // rare: multiply again and collect the passing pairs; bit
      // 16 a + 8 r + 2 nb + p = row 8 r + g of m-tile a, column
      // 8 nb + 2 tq + p, so ascending bits append tile by tile, rows g
      // before rows g + 8, lanes ascending: ascending slot order within
      // every column
      uint32_t keep = 0;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        float acc[NB][4];
        super_mma<KH, NB>(acc, x, b, a);
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) {
          const int s0 = 16 * a + 2 * nb;
          keep |= (acc[nb][0] > tn[nb][0] ? 1u : 0u) << s0;
          keep |= (acc[nb][1] > tn[nb][1] ? 1u : 0u) << (s0 + 1);
          keep |= (acc[nb][2] > tn[nb][0] ? 1u : 0u) << (s0 + 8);
          keep |= (acc[nb][3] > tn[nb][1] ? 1u : 0u) << (s0 + 9);
        }
      }
      uint32_t U = __reduce_or_sync(full, keep);
      while (U) {
        const int bit = __ffs(U) - 1;
        U &= U - 1u;
        const bool kk = (keep >> bit) & 1u;
        const unsigned m = __ballot_sync(full, kk);
        const int n = __popc(m);
        if (nq + n > kQueue) {
          drain(t, leaf, qpad, lst_d, lst_i, K, ws, lane, nq, ncol,
                (uint32_t)(sc.leaf0 * t.lcap));
          nq = 0;
        }
        if (kk)
          ws.queue[nq + __popc(m & ((1u << lane) - 1u))] =
              ((uint32_t)(S * 32 + (bit >> 4) * 16 + ((bit >> 3) & 1) * 8 + g)
               << 5) |
              (uint32_t)(((bit >> 1) & 3) * 8 + 2 * tq + (bit & 1));
        nq += n;
        kept += (unsigned long long)n;
      }
    }
  }
  cp_async_wait<0>();  // only empty groups remain; the ring is free
  if (nq)
    drain(t, leaf, qpad, lst_d, lst_i, K, ws, lane, nq, ncol,
          (uint32_t)(sc.leaf0 * t.lcap));
}

// Lane c < w.count: query id, current bound, bf16 offsets (B record) and
// the screen threshold of query column c; other lanes: an unused column.
template <int KH>
__device__ __forceinline__ void setup_column(
    const DevTree& t, const ScreenData& sc, const Item& w, int lane,
    const uint32_t* __restrict__ act, const float* __restrict__ qpad,
    const float* __restrict__ lst_d, int K, const WarpSmem& ws) {
  const float inf = __int_as_float(0x7f800000);
  uint32_t* rec = ws.rec + lane * KH * 8;
  float tneg = inf;  // unused columns keep nothing
  if (lane < w.count) {
    const uint32_t q = act[w.start + lane];
    ws.qid[lane] = q;
    const float bound = lst_d[(size_t)q * K + K - 1];
    ws.bound[lane] = bound;
    ws.flag[lane] = 0u;
    const float* qp = qpad + (size_t)q * t.Dp;
    const float* c = sc.center + (size_t)w.leaf * t.d;
    float qn = 0.f, ss = 0.f;  // |v^|^2 rounded to nearest / upward
#pragma unroll
    for (int h = 0; h < KH; ++h)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        // slots: v^ (0..d-1), then -1/2 twice against the point's norm
        const int k0 = 16 * h + 2 * j, d = t.d;
        const float a0 = k0 < d ? __fsub_rn(qp[k0], c[k0])
                                : (k0 < d + 2 ? -0.5f : 0.f);
        const float a1 = k0 + 1 < d ? __fsub_rn(qp[k0 + 1], c[k0 + 1])
                                    : (k0 + 1 < d + 2 ? -0.5f : 0.f);
        const uint32_t wd = pack_bf16(a0, a1);
        rec[h * 8 + (j < 4 ? 2 * j : 2 * (j - 4) + 1)] = wd;
        const float v0 = k0 < d ? bf16_lo(wd) : 0.f;
        const float v1 = k0 + 1 < d ? bf16_hi(wd) : 0.f;
        qn = __fmaf_rn(v0, v0, qn);
        qn = __fmaf_rn(v1, v1, qn);
        ss = __fmaf_ru(v0, v0, ss);
        ss = __fmaf_ru(v1, v1, ss);
      }
    if (isinf(bound)) {
      tneg = -inf;  // list not full: every point is a candidate
    } else {
      // T of the header comment, every step rounded upward (divisors
      // downward) so that the float result is never too small
      const float rho = 0x1p-8f * 1.0001f;  // bf16: 8 significant bits
      const float rr = __fdiv_ru(rho, __fsub_rd(1.f, rho));
      const float one_m_g = __fsub_rd(1.f, (float)(t.d + 3) * 0x1p-24f);
      const float aq = __fadd_ru(__fmul_ru(rr, __fsqrt_ru(ss)), 0x1p-123f);
      const float R =
          __fsqrt_ru(__fdiv_ru(__fadd_ru(bound, 0x1p-120f), one_m_g));
      const float Rb = __fadd_ru(__fadd_ru(R, aq), sc.bmax[w.leaf]);
      const float E = __fmul_ru(0x1p-14f, __fadd_ru(ss, sc.pnmax[w.leaf]));
      const float thr = __fsub_ru(__fadd_ru(__fmul_ru(Rb, Rb), E), qn);
      tneg = -0.5f * thr;  // exact scale
    }
  } else {
#pragma unroll
    for (int i = 0; i < KH * 8; ++i) rec[i] = 0u;
  }
  ws.tneg[lane] = tneg;
}

template <int KH>
__global__ void __launch_bounds__(kScrThreads, KH == 1 ? 3 : 2)
    warp_screen_kernel(DevTree t, ScreenData sc, const Item* __restrict__ items,
                  int item_lo, int item_hi, Counters* ctr,
                  const uint32_t* __restrict__ act,
                  const float* __restrict__ qpad, float* __restrict__ lst_d,
                  uint32_t* __restrict__ lst_i, int K) {
  extern __shared__ __align__(16) uint32_t smem_words[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpSmem ws = warp_smem<KH>(smem_words, warp, K);
  // (item_hi < 0: this round's item count, read on the device)
  const int hi = item_hi >= 0 ? item_hi : ctr->n_items;
  unsigned long long kept = 0;
  unsigned long long streamed = 0;  // operand bytes of the items' leaves
  // items are taken one at a time from a launch-wide counter: their costs
  // differ (leaf size, column blocks, rescoring), a static split leaves SMs
  // idle at the end of the launch
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(&ctr->screen_next, 1);
    it = __shfl_sync(0xffffffffu, it, 0) + item_lo;
    if (it >= hi) break;
    const Item w = items[it];
    setup_column<KH>(t, sc, w, lane, act, qpad, lst_d, K, ws);
    __syncwarp();
    const int npt = t.leaf_cnt[w.leaf];
    const int ncol = w.count;
    // (the leaf's 32-point super-tiles, 32 bytes per point and k-half)
    streamed += (unsigned long long)((npt + 31) / 32) * 32u * 32u * KH;
    switch ((ncol + 7) >> 3) {
      case 1:
        scan_leaf<KH, 1>(t, sc, w.leaf, npt, ws, lane, qpad, lst_d, lst_i, K,
                         ncol, kept);
        break;
      case 2:
        scan_leaf<KH, 2>(t, sc, w.leaf, npt, ws, lane, qpad, lst_d, lst_i, K,
                         ncol, kept);
        break;
      case 3:
        scan_leaf<KH, 3>(t, sc, w.leaf, npt, ws, lane, qpad, lst_d, lst_i, K,
                         ncol, kept);
        break;
      default:
        scan_leaf<KH, 4>(t, sc, w.leaf, npt, ws, lane, qpad, lst_d, lst_i, K,
                         ncol, kept);
        break;
    }
    if (lane < ncol && (ws.flag[lane] & 2u)) {
      const uint32_t q = ws.qid[lane];
      for (int j = 0; j < K; ++j) {
        lst_d[(size_t)q * K + j] = ws.ld[lane * K + j];
        lst_i[(size_t)q * K + j] = ws.li[lane * K + j];
      }
    }
    __syncwarp();
  }
  if (lane == 0 && kept) atomicAdd(&ctr->screen_kept, kept);
  if (lane == 0 && streamed) atomicAdd(&ctr->screen_bytes, streamed);
}

size_t screen_smem(int kh, int K) {
  return (size_t)kScrWarps * warp_words(kh, K) * 4;
}

const void* screen_kernel_for(int kh) {
  switch (kh) {
    case 1: return (const void*)warp_screen_kernel<1>;
    case 2: return (const void*)warp_screen_kernel<2>;
    case 3: return (const void*)warp_screen_kernel<3>;
    default: return nullptr;
  }
}

}  // namespace

int screen_grid_warp(int kh, int64_t lcap, int K, int sm_count) {
  // slots in a queue entry: 27 bits
  if (kh < 1 || kh > 3 || K < 1 || K > BKD_MAX_K + 1 ||
      lcap >= ((int64_t)1 << 27))
    return 0;
  const size_t smem = screen_smem(kh, K);
  const void* k = screen_kernel_for(kh);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kScrThreads,
                                                    smem) != cudaSuccess ||
      per_sm < 1)
    return 0;
  return per_sm * sm_count;
}

cudaError_t launch_screen_warp(const DevTree& t, const ScreenData& sd,
                               const Item* items, int item_lo, int item_hi,
                               Counters* ctr, const uint32_t* act,
                               const float* qpad, float* lst_d,
                               uint32_t* lst_i, int K, int grid,
                               cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  if (item_hi >= 0) {
    const int n = item_hi - item_lo;
    if (n <= 0) return cudaSuccess;
    grid = std::min(grid, (n + kScrWarps - 1) / kScrWarps);
  }
  const size_t smem = screen_smem(sd.wkh, K);
  cudaError_t e = cudaMemsetAsync(&ctr->screen_next, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  switch (sd.wkh) {
    case 1:
      warp_screen_kernel<1><<<grid, kScrThreads, smem, s>>>(
          t, sd, items, item_lo, item_hi, ctr, act, qpad, lst_d, lst_i, K);
      break;
    case 2:
      warp_screen_kernel<2><<<grid, kScrThreads, smem, s>>>(
          t, sd, items, item_lo, item_hi, ctr, act, qpad, lst_d, lst_i, K);
      break;
    case 3:
      warp_screen_kernel<3><<<grid, kScrThreads, smem, s>>>(
          t, sd, items, item_lo, item_hi, ctr, act, qpad, lst_d, lst_i, K);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace bkd
