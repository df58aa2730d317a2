// k_screen.cu -- ProcessAllBuffers with a BF16 tensor-core screen (tcgen05;
// the screen kernel selected by BKD_OPT_SCREEN_KERNEL = 1).
//
// Same candidate lists as the float32 leaf kernel (every point whose float32
// distance could still enter a query's list is scored exactly), but most
// (query, point) pairs are rejected by a cheap screen first:
//
//   v = q - c, w = x - c (c: centre of the leaf), rounded to bf16 (v^, w^);
//   s = |v^|^2 + |w^|^2 - 2 v^.w^.
//
// The tensor cores form, per (point, query) pair, in one dot product of
// 16 KH bf16 slots accumulated in fp32,
//   X = v^.w^ - (pn_hi + pn_lo) / 2 + (t_hi + t_mid + t_lo)
// where a point's row holds w^, its squared norm pn = fl32(|w^|^2) split as
// pn_hi = bf16(pn), pn_lo = bf16(pn - pn_hi) (|w^|^2 = pn_hi + pn_lo up to
// (2^-16 + 2^-24) pn), and 1, 1, 1; a query's column holds v^, -1/2, -1/2
// and its threshold t = thr / 2 split exactly into three bf16 parts.  The
// screen keeps a pair iff X > 0, i.e. iff s - |v^|^2 < thr: the threshold
// is folded into the contraction, so the epilogue only asks whether the
// largest of a row's values is positive.  Padding points (pn_hi = +inf)
// score -inf; padding columns carry t = -2^126, columns whose list is not
// full yet t = +2^126 (every point is a candidate).
//
// Safety bound.  bf16 keeps 8 significant bits, so round-to-nearest errs by
// at most 2^-8 relative; with the float32 subtraction before it, rho =
// 2^-8 (1 + 1e-4), |v^ - v| <= rho |v|, |v| <= |v^| / (1 - rho), so
//   |q - x| >= |v^ - w^| - A_q - B_x,  A_q = rho/(1-rho) |v^|,
// and B_x <= B_max, the leaf's largest such term (prepared on the host).
// The float32 distance of the exact path obeys D32 >= D (1 - g) - eta,
// g = (d+3) 2^-24, eta = 2^-120, so a point can only enter the list
// (D32 < bound) if |v^ - w^| < Rb = sqrt((bound + eta) / (1 - g)) + A_q +
// B_max, i.e. if 2 v^.w^ > |v^|^2 + |w^|^2 - Rb^2.  Then, with thr >= Rb^2
// + E - qn (qn the float32 |v^|^2),
//   X > (|v^|^2 - qn + E + pn_err) / 2,  pn_err = |w^|^2 - pn_hi - pn_lo,
// and the computed X stays positive if E covers the roundings:
//   * accumulation model: one MMA k-step (16 exact bf16 products added to
//     an fp32 accumulator c) errs by at most 2^-18 (|c| + sum |a_i b_i|), so
//     the KH chained k-halves of one pair err by at most KH 2^-18 S, S the
//     sum of the absolute products <= |v^|^2/2 + pn (1 + 2^-8) + 0.51 |thr|.
//     (A hardware property, not an IEEE rule: the MMA probe test checks it
//     on adversarial operands -- one large term and many small ones,
//     cancellation, mixed exponents within a k-half.)  Twice that (the test
//     compares 2X) is <= 2^-16.4 |v^|^2 + 2^-15.4 pn + 2^-16.3 |thr|;
//   * the norm split adds (2^-16 + 2^-24) pn, the float32 chain of |v^|^2 at
//     most d 2^-24 |v^|^2 <= 2^-19 |v^|^2;
//   * |thr| <= Rb^2 + E + qn;
// so E = 2^-13 (|v^|^2 + Rb^2) + 2^-14 pn_max + 2^-120 suffices (the last
// term covers a threshold split that underflows).  thr is formed once per
// (query, leaf) in float32 with every operation rounded toward the larger
// threshold (divisors toward the smaller).  Kept pairs are scored with the
// exact float32 chain of the leaf kernel and inserted with the same strict
// rule, so the lists hold the same k+1 smallest float32 distances as the
// float32 path, and the answers (re-check and fallback read nothing else)
// are the same.
//
// A screened round runs three kernels:
//   tc_prep_kernel      one CTA per work item (one leaf, <= 128 of its
//                       buffered queries): the item's query operand tile
//                       (v^, -1/2, -1/2, threshold parts) written to HBM;
//   tc_screen_kernel    persistent CTAs (two per SM), items taken from a
//                       launch-wide counter:
//     warp 0 (one thread)  claims items, publishes them in a small ring, and
//                          streams the query operand and the leaf's 128-point
//                          operand tiles (bulk copies, 4 KB per k-half) into
//                          a deep shared-memory ring, across item boundaries;
//     warp 1               allocates tensor memory; one thread issues, per
//                          tile, KH tcgen05.mma (M = 128 points, N = the
//                          item's queries rounded up to 16, K = 16) into one
//                          of two 128-column fp32 accumulator buffers in
//                          tensor memory -- up to four tiles of a small item
//                          side by side in one buffer -- and commits them to
//                          mbarriers (ring slot free, buffer full);
//     warps 2-9            the epilogue, two warpgroups (each half of a
//                          buffer's column groups): per buffer read the
//                          accumulator (tcgen05.ld, row = point, column =
//                          query), take the largest value of each row over
//                          each group of 16 columns with three-input max,
//                          hand the buffer back, and append the rare (point,
//                          group) pairs with a positive value to the item's
//                          survivor segment in HBM;
//   tc_rescore_kernel   scores the survivors exactly (float32 chain of the
//                       leaf kernel) against the 16 queries of their group
//                       and inserts them into the lists; an item whose
//                       segment overflowed goes to the float32 leaf kernel.
// Every wait is bounded: a wait that runs out sets kErrTimeout, every role
// then leaves, copies and MMAs in flight are waited for (bounded), and the
// tensor memory is released.
#include <cuda_bf16.h>

#include <algorithm>

#include "bkd.h"
#include "bkd_internal.h"
#include "k_leaf.cuh"

namespace bkd {
namespace {

constexpr int kEpiThreads = 256;              // 2 x 4 epilogue warps
constexpr int kThreads = 64 + kEpiThreads;    // + producer warp + MMA warp
constexpr int kItemRing = 8;                  // published items in flight
constexpr int kBops = 4;                      // query-operand buffers
constexpr int kClaim = 4;                     // items claimed at a time
constexpr uint32_t kAccCols = 128;            // tensor-memory columns per acc
constexpr uint32_t kTmemCols = 2 * kAccCols;  // two accumulators

// Point tiles in flight per CTA: about three leaves of 1,024 points, so
// that the copies of the next items hide the HBM latency.
__host__ __device__ constexpr int ring_stages(int kh) {
  return kh == 1 ? 20 : (kh == 2 ? 8 : 6);
}
__host__ __device__ constexpr uint32_t tile_bytes(int kh) {
  return 4096u * (uint32_t)kh;
}
// Accumulator columns of one point tile of an item with G groups of 16
// query columns: rounded up to 32, so that 128 / slot_cols tiles share an
// accumulator buffer (4 for G <= 2, 2 for G <= 4, else 1).
__host__ __device__ constexpr uint32_t slot_cols(int G) {
  return G <= 2 ? 32u : (G <= 4 ? 64u : 128u);
}

// Shared-memory layout (byte offsets into the dynamic shared memory).
struct Layout {
  uint32_t ring, bop, items, bars, misc, total;
};

__host__ __device__ inline uint32_t take(uint32_t& o, uint32_t bytes,
                                         uint32_t align) {
  o = (o + align - 1) / align * align;
  const uint32_t r = o;
  o += bytes;
  return r;
}

__host__ __device__ inline Layout layout_of(int kh) {
  Layout L;
  uint32_t o = 0;
  L.ring = take(o, ring_stages(kh) * tile_bytes(kh), 1024);
  L.bop = take(o, kBops * tile_bytes(kh), 1024);  // query operands
  L.items = take(o, kItemRing * 16, 16);
  L.bars = take(o,
                (2 * ring_stages(kh) + 5 + 2 * kBops + 2 * kItemRing) * 8, 8);
  L.misc = take(o, 32, 16);
  L.total = o;
  return L;
}

// ----------------------------------------------------------- primitives
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// The same test, but a thread whose phase is not complete yet is suspended
// by the hardware until it completes (or about a millisecond passes)
// instead of returning at once: waiting threads take no issue slots from
// the working ones.
__device__ __forceinline__ bool bar_try_suspend(uint32_t bar,
                                                uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of `bar`; false once the CTA aborted or the wait
// ran out (~2^31 cycles: then it aborts the CTA and reports the timeout).
__device__ __noinline__ bool bar_wait_slow(uint32_t bar, uint32_t parity,
                                           volatile int* abort,
                                           Counters* ctr) {
  const long long t0 = clock64();
  for (;;) {
    if (bar_try_suspend(bar, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > (1ll << 31)) {
      *abort = 1;
      atomicOr(&ctr->err, kErrTimeout);
      return false;
    }
  }
}
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity,
                                         volatile int* abort, Counters* ctr) {
  return bar_try(bar, parity) || bar_wait_slow(bar, parity, abort, ctr);
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor of an operand tile in the layout of
// screen_row_offset (no swizzle, K-major): start address, leading-dimension
// byte offset (K direction: 128), stride-dimension byte offset (8-row
// groups: 256 kh), descriptor version 1.
__device__ __forceinline__ uint64_t op_desc(uint32_t saddr, int kh) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) |
         ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(((uint32_t)kh * 256u) >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: bf16 A and B, fp32 accumulator,
// both K-major, M = 128, N = n (multiple of 16, <= 256).
__device__ __forceinline__ uint32_t mma_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
      "[%0];" ::"r"(bar)
      : "memory");
}

// 16 / 32 consecutive accumulator columns of this thread's lane, waited for
// inside the same statement (so no use can be scheduled before the wait).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, "
      "%7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
        "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]),
        "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Two groups of 16 columns at arbitrary column addresses, one wait.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t taddr2,
                                        float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, "
      "%7, %8, %9, %10, %11, %12, %13, %14, %15}, [%32];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, "
      "%22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%33];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
        "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]),
        "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr), "r"(taddr2)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// max(a, b, c) (three-input float max of sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

__device__ __forceinline__ float bf16_value(uint16_t h) {
  return __uint_as_float((uint32_t)h << 16);
}
__device__ __forceinline__ uint16_t bf16_bits(float f) {
  const __nv_bfloat16 b = __float2bfloat16_rn(f);
  return *reinterpret_cast<const uint16_t*>(&b);
}

// ------------------------------------------------------------ prep kernel
// The query operand of every work item of the round, written to HBM in the
// layout of an operand tile (screen_row_offset, 128 rows): row e is query
// column e of the item (v^, -1/2, -1/2, the threshold split into three
// bf16 parts), rows e >= count padding columns (threshold -2^126: never
// kept).  A column whose list is not full yet (bound +inf: every point may
// enter) gets threshold +2^126.  One CTA of 128 threads per item, items
// read from the device's count of the round.
template <int KH>
__global__ void __launch_bounds__(128)
    tc_prep_kernel(DevTree t, ScreenData sc, const Item* __restrict__ items,
                const Counters* __restrict__ ctr,
                const uint32_t* __restrict__ act,
                const float* __restrict__ qpad,
                const float* __restrict__ lst_d, int K,
                uint8_t* __restrict__ bop) {
  const int n_items = ctr->n_items;
  const int e = threadIdx.x;
  const int d = t.d;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const Item w = items[it];
    uint16_t th = 0xfe80, tm = 0, tl = 0;  // -2^126: never kept
    float vq[16 * KH];
#pragma unroll
    for (int i = 0; i < 16 * KH; ++i) vq[i] = 0.f;
    if (e < w.count) {
      const uint32_t q = act[w.start + e];
      const float bound = lst_d[(size_t)q * K + K - 1];
      const float* qp = qpad + (size_t)q * t.Dp;
      const float* c = sc.center + (size_t)w.leaf * d;
      float qn = 0.f, ss = 0.f;  // |v^|^2 rounded to nearest / upward
#pragma unroll
      for (int i = 0; i < 16 * KH; ++i)
        if (i < d) {
          const float v = bf16_value(bf16_bits(__fsub_rn(qp[i], c[i])));
          vq[i] = v;
          qn = __fmaf_rn(v, v, qn);
          ss = __fmaf_ru(v, v, ss);
        }
      if (isinf(bound)) {
        th = 0x7e80;  // +2^126: the list is not full, every point may enter
      } else {
        // thr of the header comment, every step rounded upward (divisors
        // downward) so that the float result is never too small
        const float rho = 0x1p-8f * 1.0001f;  // bf16: 8 significant bits
        const float rr = __fdiv_ru(rho, __fsub_rd(1.f, rho));
        const float one_m_g = __fsub_rd(1.f, (float)(d + 3) * 0x1p-24f);
        const float aq = __fadd_ru(__fmul_ru(rr, __fsqrt_ru(ss)), 0x1p-123f);
        const float R =
            __fsqrt_ru(__fdiv_ru(__fadd_ru(bound, 0x1p-120f), one_m_g));
        const float Rb = __fadd_ru(__fadd_ru(R, aq), sc.bmax[w.leaf]);
        const float Rb2 = __fmul_ru(Rb, Rb);
        const float E = __fadd_ru(
            __fmul_ru(0x1p-13f, __fadd_ru(ss, Rb2)),
            __fadd_ru(__fmul_ru(0x1p-14f, sc.pnmax[w.leaf]), 0x1p-120f));
        const float thr = __fsub_ru(__fadd_ru(Rb2, E), qn);
        // t = thr / 2 split into three bf16 parts; each remainder is exact
        // in float32 (it keeps at most 16, then 8 significant bits)
        const float tt = 0.5f * thr;
        th = bf16_bits(tt);
        const float r1 = __fsub_rn(tt, bf16_value(th));
        tm = bf16_bits(r1);
        const float r2 = __fsub_rn(r1, bf16_value(tm));
        tl = bf16_bits(r2);
      }
    }
    // slots: v^ (0..d-1), -1/2, -1/2 against the norm split, the threshold;
    // only the item's columns rounded up to 16 (the MMA's N) are written:
    // the screen reads no other row of the tile
    if (e >= ((w.count + 15) & ~15)) continue;
    uint8_t* tile = bop + (size_t)it * tile_bytes(KH);
#pragma unroll
    for (int kg = 0; kg < 2 * KH; ++kg) {
      uint32_t wv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint16_t h2[2];
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          const int slot = 8 * kg + 2 * j + x;
          h2[x] = slot < d        ? bf16_bits(vq[slot < 16 * KH ? slot : 0])
                  : slot < d + 2  ? (uint16_t)0xbf00
                  : slot == d + 2 ? th
                  : slot == d + 3 ? tm
                  : slot == d + 4 ? tl
                                  : (uint16_t)0;
        }
        wv[j] = (uint32_t)h2[0] | ((uint32_t)h2[1] << 16);
      }
      *reinterpret_cast<uint4*>(tile + screen_row_offset(e, kg, KH)) =
          make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
  }
}

// ---------------------------------------------------------- screen kernel
// The screen's view of its dynamic shared memory.
struct Smem {
  uint8_t* base;
  uint32_t base_u32;
  Layout L;
  int S;
  __device__ uint32_t ring_u32(int s, int kh) const {
    return base_u32 + L.ring + (uint32_t)s * tile_bytes(kh);
  }
  __device__ uint32_t bop_u32(int g, int kh) const {
    return base_u32 + L.bop + (uint32_t)g * tile_bytes(kh);
  }
  __device__ uint32_t bar(int i) const { return base_u32 + L.bars + 8u * i; }
  __device__ uint32_t afull(int s) const { return bar(s); }
  __device__ uint32_t aempty(int s) const { return bar(S + s); }
  __device__ uint32_t accfull(int b) const { return bar(2 * S + b); }
  __device__ uint32_t accempty(int b) const { return bar(2 * S + 2 + b); }
  __device__ uint32_t bfull(int g) const { return bar(2 * S + 4 + g); }
  __device__ uint32_t bempty(int g) const {
    return bar(2 * S + 4 + kBops + g);
  }
  __device__ uint32_t itemfull(int i) const {
    return bar(2 * S + 4 + 2 * kBops + i);
  }
  __device__ uint32_t itemempty(int i) const {
    return bar(2 * S + 4 + 2 * kBops + kItemRing + i);
  }
  __device__ uint32_t drain() const {
    return bar(2 * S + 4 + 2 * kBops + 2 * kItemRing);
  }
  __device__ int4* items() const {
    return reinterpret_cast<int4*>(base + L.items);
  }
  // misc words: [0] tensor-memory base, [1] abort
  __device__ uint32_t* misc() const {
    return reinterpret_cast<uint32_t*>(base + L.misc);
  }
};

// Survivors of the screen: per work item and epilogue warp a sub-segment
// of kWarpCap entries (point index in the leaf << 3 | group of 16 query
// columns: the point passed the screen for at least one query of the
// group) and its count (a count above kWarpCap: the sub-segment
// overflowed; the item is scored by the float32 leaf kernel instead).
constexpr int kEpiWarps = kEpiThreads / 32;
constexpr int kWarpCap = 128;
constexpr int kSegCap = kEpiWarps * kWarpCap;  // entries per item

template <int KH>
__global__ void __launch_bounds__(kThreads, 2)
    tc_screen_kernel(DevTree t, ScreenData sc, const Item* __restrict__ items,
                  int item_lo, int item_hi, Counters* ctr,
                  const uint8_t* __restrict__ bop_g,
                  uint32_t* __restrict__ seg, int32_t* __restrict__ seg_cnt) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem sm;
  sm.base = smem_raw;
  sm.base_u32 = (uint32_t)__cvta_generic_to_shared(smem_raw);
  sm.L = layout_of(KH);
  sm.S = ring_stages(KH);
  const int S = sm.S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort = reinterpret_cast<volatile int*>(sm.misc() + 1);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(sm.afull(s), 1);
      mbar_init(sm.aempty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(sm.accfull(b), 1);
      mbar_init(sm.accempty(b), kEpiThreads);
    }
    for (int g = 0; g < kBops; ++g) {
      mbar_init(sm.bfull(g), 1);
      mbar_init(sm.bempty(g), 1);
    }
    for (int i = 0; i < kItemRing; ++i) {
      mbar_init(sm.itemfull(i), 1);
      mbar_init(sm.itemempty(i), 1 + kEpiThreads);
    }
    mbar_init(sm.drain(), 1);
    for (int i = 1; i < 8; ++i) sm.misc()[i] = 0;
    mbar_init_fence();
  }
  if (warp == 1) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::
            "r"(sm.base_u32 + sm.L.misc),
        "r"(kTmemCols)
        : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;"
                 ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.misc()[0];
  const int64_t tiles = sc.tiles;
  const uint8_t* words = reinterpret_cast<const uint8_t*>(sc.words);

  if (warp == 0) {
    // ------------------------------------------------------- producer
    // (item_hi < 0: this round's item count, read on the device)
    const int hi = item_hi >= 0 ? item_hi : ctr->n_items;
    if (lane == 0) {
      uint32_t c = 0;  // point tiles issued
      unsigned long long bop_bytes = 0;  // query operand bytes loaded
      uint32_t last[20];  // last tile issued into each ring slot + 1
      uint32_t lastb[kBops];  // last item (+1) whose operand went into each
                              // query-operand buffer
      for (int s = 0; s < S; ++s) last[s] = 0;
      for (int g = 0; g < kBops; ++g) lastb[g] = 0;
      // items are claimed kClaim at a time; their descriptors and leaf sizes
      // are loaded together (one memory latency per claim)
      Item wq[kClaim];
      int nq[kClaim];
      int have = 0, at = 0, first = 0;
      int n = 0;
      for (;; ++n) {
        if (at == have) {
          first = atomicAdd(&ctr->screen_next, kClaim) + item_lo;
          have = max(0, min(kClaim, hi - first));
          at = 0;
#pragma unroll
          for (int j = 0; j < kClaim; ++j)
            if (j < have) wq[j] = items[first + j];
#pragma unroll
          for (int j = 0; j < kClaim; ++j)
            if (j < have) nq[j] = t.leaf_cnt[wq[j].leaf];
        }
        const int ir = n % kItemRing, g = n % kBops;
        if (!bar_wait(sm.itemempty(ir), ((n / kItemRing) & 1) ^ 1, abort,
                      ctr))
          break;
        if (have == 0) {
          sm.items()[ir] = make_int4(-1, 0, 0, 0);
          bar_arrive(sm.itemfull(ir));
          break;
        }
        Item w = wq[0];
        int np = nq[0];
#pragma unroll
        for (int j = 1; j < kClaim; ++j)
          if (j == at) {
            w = wq[j];
            np = nq[j];
          }
        const int it = first + at;
        ++at;
        const int nt = (np + kScreenRows - 1) / kScreenRows;
        sm.items()[ir] = make_int4(w.leaf, it, w.count, nt);
        bar_arrive(sm.itemfull(ir));
        // the item's query operand, once the MMAs of the item kBops before
        // are done with the buffer
        if (!bar_wait(sm.bempty(g), ((n / kBops) & 1) ^ 1, abort, ctr))
          break;
        // (its first 16 G rows: the MMA's N columns, contiguous in the
        // operand layout)
        const uint32_t bbytes = 512u * KH * (uint32_t)((w.count + 15) >> 4);
        bulk_load(sm.bop_u32(g, KH), bop_g + (size_t)it * tile_bytes(KH),
                  bbytes, sm.bfull(g));
        bop_bytes += bbytes;
        lastb[g] = (uint32_t)n + 1;
        const uint8_t* src = words + (size_t)w.leaf * tiles * tile_bytes(KH);
        bool ok = true;
        for (int ti = 0; ti < nt; ++ti, ++c) {
          const int s = c % S;
          if (!bar_wait(sm.aempty(s), ((c / S) & 1) ^ 1, abort, ctr)) {
            ok = false;
            break;
          }
          bulk_load(sm.ring_u32(s, KH), src + (size_t)ti * tile_bytes(KH),
                    tile_bytes(KH), sm.afull(s));
          last[s] = c + 1;
        }
        if (!ok) break;
      }
      if (c)
        atomicAdd(&ctr->screen_bytes,
                  (unsigned long long)c * tile_bytes(KH) + bop_bytes);
      // copies still in flight land before the CTA leaves
      for (int s = 0; s < S; ++s)
        if (last[s]) {
          const uint32_t cl = last[s] - 1;
          const long long t0 = clock64();
          while (!bar_try(sm.afull(s), (cl / S) & 1) &&
                 clock64() - t0 < (1ll << 31)) {
          }
        }
      for (int g = 0; g < kBops; ++g)
        if (lastb[g]) {
          const uint32_t nl = lastb[g] - 1;
          const long long t0 = clock64();
          while (!bar_try(sm.bfull(g), (nl / kBops) & 1) &&
                 clock64() - t0 < (1ll << 31)) {
          }
        }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t c = 0;   // tiles consumed
      uint32_t cb = 0;  // accumulator buffers filled
      bool issued = false;
      for (int n = 0;; ++n) {
        const int ir = n % kItemRing, g = n % kBops;
        if (!bar_wait(sm.itemfull(ir), (n / kItemRing) & 1, abort, ctr))
          break;
        const int4 dsc = sm.items()[ir];
        bar_arrive(sm.itemempty(ir));
        if (dsc.x < 0) break;
        if (!bar_wait(sm.bfull(g), (n / kBops) & 1, abort, ctr)) break;
        const int G = (dsc.z + 15) >> 4;
        const uint32_t sw = slot_cols(G);
        const int T = (int)(kAccCols / sw);
        const uint32_t idesc = mma_idesc(16 * G);
        const uint32_t bop = sm.bop_u32(g, KH);
        bool ok = true;
        for (int t0 = 0; ok && t0 < dsc.w; t0 += T, ++cb) {
          const int b = cb & 1;
          if (!bar_wait(sm.accempty(b), ((cb >> 1) & 1) ^ 1, abort, ctr)) {
            ok = false;
            break;
          }
          const int nk = min(T, dsc.w - t0);
          for (int k = 0; k < nk; ++k, ++c) {
            const int s = c % S;
            if (!bar_wait(sm.afull(s), (c / S) & 1, abort, ctr)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = sm.ring_u32(s, KH);
            const uint32_t d = tmem + (uint32_t)b * kAccCols + (uint32_t)k * sw;
#pragma unroll
            for (int h = 0; h < KH; ++h)
              tc_mma(d, op_desc(a0 + 256u * h, KH), op_desc(bop + 256u * h, KH),
                     idesc, h > 0 ? 1u : 0u);
            tc_commit(sm.aempty(s));
            issued = true;
          }
          if (ok) tc_commit(sm.accfull(b));
        }
        tc_commit(sm.bempty(g));  // the query operand buffer is free
        if (!ok) break;
      }
      if (issued) {
        // every MMA issued has completed before the CTA leaves
        tc_commit(sm.drain());
        const long long t0 = clock64();
        while (!bar_try(sm.drain(), 0) && clock64() - t0 < (1ll << 31)) {
        }
      }
    }
  } else {
    // ------------------------------------------------------- epilogue
    // Two warpgroups: warp w reads tensor-memory lanes 32 (w % 4) .. (its
    // accumulator rows = points).  An accumulator buffer holds the tiles of
    // T = 128 / slot_cols(G) consecutive point tiles of the item side by
    // side (G groups of 16 query columns each): of its groups warpgroup 0
    // takes the first half (rounded up), warpgroup 1 the rest.  Per buffer a
    // thread takes the largest value of its row over each of its groups; a
    // (point, group) pair with a positive value goes to the warp's
    // sub-segment of the item (a warp-uniform count in registers: no
    // atomics).  The rescoring kernel then scores that point exactly
    // against every query of the group.  The warps run independently; a
    // failed wait (abort or timeout) makes the warp leave.
    const int quarter = warp & 3;  // tensor-memory lanes 32 quarter ..
    const int half = (warp - 2) >> 2;
    const int ew = warp - 2;       // epilogue warp 0 .. kEpiWarps - 1
    const int row = 32 * quarter + lane;
    const unsigned below = (1u << lane) - 1u;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
    uint32_t cb = 0;
    unsigned long long kept = 0;
    for (int n = 0;; ++n) {
      const int ir = n % kItemRing;
      if (!__all_sync(0xffffffffu, bar_wait(sm.itemfull(ir),
                                             (n / kItemRing) & 1, abort, ctr)))
        break;
      const int4 dsc = sm.items()[ir];
      bar_arrive(sm.itemempty(ir));
      if (dsc.x < 0) break;
      const int it = dsc.y, nt = dsc.w;
      const int G = (dsc.z + 15) >> 4;  // column groups of the item
      const uint32_t sw = slot_cols(G);
      const int T = (int)(kAccCols / sw);
      uint32_t* out = seg + ((size_t)it * kEpiWarps + ew) * kWarpCap;
      uint32_t cnt = 0;  // entries of this warp for the item
      bool ok = true;
      for (int t0 = 0; t0 < nt; t0 += T, ++cb) {
        const int b = cb & 1;
        if (!__all_sync(0xffffffffu,
                        bar_wait(sm.accfull(b), (cb >> 1) & 1, abort, ctr))) {
          ok = false;
          break;
        }
        // this warp's groups [j0, j1) of the buffer's nk G groups (group
        // j: tile j / G of the buffer, column group j % G; both walked
        // incrementally from (k0, g0), no division in the loop)
        const int GT = min(T, nt - t0) * G, gh = (GT + 1) >> 1;
        const int j0 = half ? gh : 0, j1 = half ? GT : gh;
        const int k0 = half ? gh / G : 0, g0 = half ? gh - k0 * G : 0;
        const uint32_t ta = lane_base + (uint32_t)b * kAccCols;
        uint32_t grp = 0u;  // bit j - j0: group j passes for this row
        tc_fence_after();
        int kk = k0, gg = g0;  // (tile, group) of group j
#pragma unroll 1
        for (int j = j0; j < j1; j += 2) {
          float v[32];
          const uint32_t a0 = ta + (uint32_t)kk * sw + 16u * (uint32_t)gg;
          if (++gg == G) {
            gg = 0;
            ++kk;
          }
          if (j + 1 < j1) {
            tc_ld32(a0, ta + (uint32_t)kk * sw + 16u * (uint32_t)gg, v);
            if (++gg == G) {
              gg = 0;
              ++kk;
            }
          } else {
            tc_ld16(a0, v);
#pragma unroll
            for (int i = 16; i < 32; ++i) v[i] = -INFINITY;
          }
          float m[10];
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const float* x = v + 16 * h2;
#pragma unroll
            for (int i = 0; i < 5; ++i)
              m[5 * h2 + i] = fmax3(x[3 * i], x[3 * i + 1], x[3 * i + 2]);
          }
          const float lo = fmax3(fmax3(m[0], m[1], m[2]), m[3],
                                 fmaxf(m[4], v[15]));
          const float hi = fmax3(fmax3(m[5], m[6], m[7]), m[8],
                                 fmaxf(m[9], v[31]));
          grp |= (lo > 0.f ? 1u : 0u) << (j - j0);
          grp |= (hi > 0.f ? 1u : 0u) << (j - j0 + 1);
        }
        tc_fence_before();
        bar_arrive(sm.accempty(b));
        // rare: (row, group) pairs that pass, one entry each
        if (__any_sync(0xffffffffu, grp != 0u)) {
          int ks = k0, gs = g0;
          for (int j = j0; j < j1; ++j) {
            const bool mine = (grp >> (j - j0)) & 1u;
            const unsigned pass = __ballot_sync(0xffffffffu, mine);
            if (mine) {
              const uint32_t u = (uint32_t)((t0 + ks) * kScreenRows + row);
              const uint32_t at = cnt + (uint32_t)__popc(pass & below);
              if (at < (uint32_t)kWarpCap)
                out[at] = (u << 3) | (uint32_t)gs;
              kept += 16;
            }
            cnt += (uint32_t)__popc(pass);
            if (++gs == G) {
              gs = 0;
              ++ks;
            }
          }
        }
      }
      if (lane == 0) seg_cnt[(size_t)it * kEpiWarps + ew] = (int32_t)cnt;
      if (!ok) break;
    }
    if (kept) atomicAdd(&ctr->screen_kept, kept);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::
                     "r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// --------------------------------------------------------- rescore kernel
// Exact rescoring of the survivors.  One warp per unit (work item, block of
// 32 query columns): lane j owns query column 32 b + j of the item.  The
// warp reads its queries' list bounds (the last list entry), then walks the
// item's segment 32 entries at a time: the entries of its two 16-column
// groups are compacted and their points staged in the warp's shared memory
// (one coalesced load per point coordinate), and every lane scores the
// staged points of its own group with the float32 chain of the leaf kernel.
// A point below the bound is inserted (strict rule) into the list, which is
// read from HBM on the first insertion and written back at the end.  An
// item whose segment overflowed is handed to the float32 leaf kernel
// (appended to `ovf`) and not touched here.  Units are taken grid-stride
// over the device's item count of the round.
constexpr int kRescoreWarps = 8;

template <int D>
__global__ void __launch_bounds__(32 * kRescoreWarps)
    tc_rescore_kernel(DevTree t, const Item* __restrict__ items,
                   Counters* ctr, const uint32_t* __restrict__ act,
                   const float* __restrict__ qpad, float* __restrict__ lst_d,
                   uint32_t* __restrict__ lst_i, int K,
                   const uint32_t* __restrict__ seg,
                   const int32_t* __restrict__ seg_cnt,
                   Item* __restrict__ ovf) {
  constexpr int kStride = D + 1;  // staged point: D coordinates + entry
  __shared__ float stage[kRescoreWarps][32 * kStride];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* st = stage[wib];
  const int64_t n_units = 4 * (int64_t)ctr->n_items;
  const int64_t nw = (int64_t)gridDim.x * kRescoreWarps;
  const unsigned below = (1u << lane) - 1u;
  unsigned long long queued = 0, overflow = 0;
  for (int64_t u = (int64_t)blockIdx.x * kRescoreWarps + wib; u < n_units;
       u += nw) {
    const int it = (int)(u >> 2), cb = (int)(u & 3);
    // lanes 0 .. kEpiWarps - 1: the item's sub-segment counts
    const int cl = lane < kEpiWarps ? seg_cnt[(size_t)it * kEpiWarps + lane]
                                    : 0;
    const int total = __reduce_add_sync(0xffffffffu, max(cl, 0));
    if (total == 0) continue;
    const Item w = items[it];
    if (cb * 32 >= w.count) continue;
    if (__any_sync(0xffffffffu, cl > kWarpCap)) {
      // the float32 leaf kernel takes items of at most kPipeTile queries
      if (cb == 0 && lane == 0) {
        const int parts = (w.count + kPipeTile - 1) / kPipeTile;
        const int at = atomicAdd(&ctr->screen_ovf_items, parts);
        for (int j = 0; j < parts; ++j)
          ovf[at + j] = Item{w.leaf, w.start + j * kPipeTile,
                             min(kPipeTile, w.count - j * kPipeTile), 0};
        ++overflow;
      }
      continue;
    }
    if (cb == 0 && lane == 0) queued += (unsigned long long)total;
    const int col = cb * 32 + lane;
    const bool valid = col < w.count;
    const uint32_t q = valid ? act[w.start + col] : 0u;
    float qr[D];
#pragma unroll
    for (int i = 0; i < D; ++i) qr[i] = valid ? qpad[(size_t)q * D + i] : 0.f;
    float bound = valid ? lst_d[(size_t)q * K + K - 1] : -INFINITY;
    const uint32_t my_group = (uint32_t)(col >> 4);
    const uint32_t slot0 = (uint32_t)((int64_t)w.leaf * t.lcap);
    float Ld[BKD_MAX_K + 1];
    uint32_t Li[BKD_MAX_K + 1];
    bool loaded = false, changed = false;
    // every sub-segment may hold entries of this unit's groups 2 cb and
    // 2 cb + 1 (the screen splits a buffer's tiles and groups between its
    // warpgroups)
    for (int e = 0; e < kEpiWarps; ++e) {
      const int cnt = __shfl_sync(0xffffffffu, cl, e);
      const uint32_t* sg = seg + ((size_t)it * kEpiWarps + e) * kWarpCap;
      for (int base = 0; base < cnt; base += 32) {
        uint32_t en = 0u;
        bool rel = false;
        if (base + lane < cnt) {
          en = sg[base + lane];
          // (entries of a leaf's padding rows never pass; the bound on the
          // point index keeps a stale count from reading past the leaf)
          rel = ((en & 7u) >> 1) == (uint32_t)cb && (en >> 3) < t.lcap;
        }
        const unsigned m = __ballot_sync(0xffffffffu, rel);
        if (!m) continue;
        if (rel) {
          const int r = __popc(m & below);
          const uint32_t slot = slot0 + (en >> 3);
          const float* quad = t.pts + (size_t)(slot >> 2) * 4 * D + (slot & 3);
          float* dst = st + r * kStride;
#pragma unroll
          for (int i = 0; i < D; ++i) dst[i] = quad[4 * i];
          dst[D] = __uint_as_float(en);
        }
        __syncwarp();
        const int nr = __popc(m);
        for (int r = 0; r < nr; ++r) {
          const float* sp = st + r * kStride;
          const uint32_t er = __float_as_uint(sp[D]);
          if ((er & 7u) != my_group) continue;
          float dd = __fsub_rn(qr[0], sp[0]);
          float dv = __fmul_rn(dd, dd);
#pragma unroll
          for (int i = 1; i < D; ++i) {
            dd = __fsub_rn(qr[i], sp[i]);
            dv = __fmaf_rn(dd, dd, dv);
          }
          if (dv < bound) {
            if (!loaded) {
              for (int j = 0; j < K; ++j) {
                Ld[j] = lst_d[(size_t)q * K + j];
                Li[j] = lst_i[(size_t)q * K + j];
              }
              loaded = true;
            }
            int pos = K - 1;
            while (pos > 0 && Ld[pos - 1] > dv) {
              Ld[pos] = Ld[pos - 1];
              Li[pos] = Li[pos - 1];
              --pos;
            }
            Ld[pos] = dv;
            Li[pos] = slot0 + (er >> 3);
            bound = Ld[K - 1];
            changed = true;
          }
        }
        __syncwarp();
      }
    }
    if (changed)
      for (int j = 0; j < K; ++j) {
        lst_d[(size_t)q * K + j] = Ld[j];
        lst_i[(size_t)q * K + j] = Li[j];
      }
  }
  if (queued || overflow) {
    atomicAdd(&ctr->screen_queued, queued);
    atomicAdd(&ctr->screen_overflow, overflow);
  }
}

using RescoreFn = void (*)(DevTree, const Item*, Counters*, const uint32_t*,
                           const float*, float*, uint32_t*, int,
                           const uint32_t*, const int32_t*, Item*);
RescoreFn rescore_for(int dp) {
  switch (dp) {
#define BKD_RESCORE_CASE(D) \
  case D:                   \
    return tc_rescore_kernel<D>;
    BKD_DIMS(BKD_RESCORE_CASE)
#undef BKD_RESCORE_CASE
    default: return nullptr;
  }
}

const void* screen_kernel_for(int kh) {
  switch (kh) {
    case 1: return (const void*)tc_screen_kernel<1>;
    case 2: return (const void*)tc_screen_kernel<2>;
    case 3: return (const void*)tc_screen_kernel<3>;
    default: return nullptr;
  }
}

// Dynamic shared memory of a launch: the layout, raised if needed so that
// at most two CTAs share an SM (two accumulator pairs fill its tensor
// memory: an allocation never has to wait for another CTA).
size_t screen_smem(int kh) {
  const size_t need = layout_of(kh).total;
  return std::max<size_t>(need, 80 * 1024);
}

// ------------------------------------------------------------ MMA probe
// One CTA per instance: D = A Bt^T with A 128 x 16 kh, Bt n x 16 kh (bf16,
// row-major), through the screen's operand layout, descriptors, KH chained
// MMAs into tensor memory and tcgen05.ld.
template <int KH>
__global__ void __launch_bounds__(128)
    umma_probe_kernel(int n, const uint16_t* __restrict__ A,
                      const uint16_t* __restrict__ Bt, float* __restrict__ D,
                      Counters* ctr) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(smem_raw);
  const uint32_t aoff = 0, boff = tile_bytes(KH),
                 baroff = boff + 2 * tile_bytes(KH), toff = baroff + 8;
  const int inst = blockIdx.x, tid = threadIdx.x, warp = tid >> 5;
  const uint16_t* a = A + (size_t)inst * 128 * 16 * KH;
  const uint16_t* bt = Bt + (size_t)inst * n * 16 * KH;
  for (int kg = 0; kg < 2 * KH; ++kg) {
    *reinterpret_cast<uint4*>(smem_raw + aoff +
                              screen_row_offset(tid, kg, KH)) =
        *reinterpret_cast<const uint4*>(a + (size_t)tid * 16 * KH + 8 * kg);
    for (int r = tid; r < n; r += 128)
      *reinterpret_cast<uint4*>(smem_raw + boff +
                                screen_row_offset(r, kg, KH)) =
          *reinterpret_cast<const uint4*>(bt + (size_t)r * 16 * KH + 8 * kg);
  }
  if (tid == 0) {
    mbar_init(base + baroff, 1);
    mbar_init_fence();
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::
            "r"(base + toff),
        "r"(256u)
        : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;"
                 ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<uint32_t*>(smem_raw + toff);
  if (tid == 0) {
    for (int h = 0; h < KH; ++h)
      tc_mma(tmem, op_desc(base + aoff + 256u * h, KH),
             op_desc(base + boff + 256u * h, KH), mma_idesc(n),
             h > 0 ? 1u : 0u);
    tc_commit(base + baroff);
  }
  const long long t0 = clock64();
  bool ok = true;
  while (!bar_try(base + baroff, 0)) {
    if (clock64() - t0 > (1ll << 31)) {
      ok = false;
      break;
    }
  }
  if (!ok) {
    if (tid == 0) atomicOr(&ctr->err, kErrTimeout);
  } else {
    tc_fence_after();
    const uint32_t lb = tmem + ((uint32_t)(32 * warp) << 16);
    for (int c0 = 0; c0 < n; c0 += 16) {
      float v[16];
      tc_ld16(lb + (uint32_t)c0, v);
      for (int i = 0; i < 16; ++i)
        D[((size_t)inst * 128 + tid) * n + c0 + i] = v[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::
                     "r"(tmem),
                 "r"(256u)
                 : "memory");
}

}  // namespace

int screen_grid(const ScreenData& sd, int Dp, int64_t lcap, int K,
                int sm_count) {
  if (!sd.on()) return 0;
  if (sd.kind == 0) return screen_grid_warp(sd.wkh, lcap, K, sm_count);
  const int kh = sd.kh;
  if (kh < 1 || kh > 3 || Dp < 1 || K < 1 || K > BKD_MAX_K + 1 ||
      lcap >= ((int64_t)1 << 24))
    return 0;
  const size_t smem = screen_smem(kh);
  const void* k = screen_kernel_for(kh);
  if (smem > 227 * 1024 ||
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                           100) != cudaSuccess)
    return 0;
  // CTAs per SM: shared memory (with the per-block reservation), registers
  // and tensor memory (512 columns per SM, kTmemCols per CTA)
  int dev = 0, smem_sm = 0, smem_rsv = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm,
                             cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                             dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_rsv,
                             cudaDevAttrReservedSharedMemoryPerBlock,
                             dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k) != cudaSuccess)
    return 0;
  const int by_smem = smem_sm / (int)(smem + smem_rsv);
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
  const int by_regs = 65536 / (regs_warp * (kThreads / 32));
  const int per_sm =
      std::min(std::min(by_smem, by_regs), (int)(512 / kTmemCols));
  if (per_sm < 1) return 0;
  return per_sm * sm_count;
}

int64_t screen_seg_cap() { return kSegCap; }
int64_t screen_cnt_per_item() { return kEpiWarps; }

cudaError_t launch_screen(const DevTree& t, const ScreenData& sd,
                          const Item* items, int n_items, Counters* ctr,
                          const uint32_t* act, const float* qpad,
                          float* lst_d, uint32_t* lst_i, int K, int grid,
                          const ScreenWork& w, int cap, int leaf_grid,
                          int sm_count, cudaStream_t s) {
  if (n_items == 0 || grid <= 0) return cudaSuccess;
  if (sd.kind == 0)
    return launch_screen_warp(t, sd, items, 0, n_items, ctr, act, qpad, lst_d,
                              lst_i, K, grid, s);
  if (n_items > 0) grid = std::min(grid, n_items);
  const int aux = n_items > 0 ? std::min(n_items, sm_count * 16)
                              : sm_count * 16;
  // rescoring: four units per item, kRescoreWarps units per CTA
  const int64_t units = 4 * (int64_t)std::max(n_items, 0);
  const int rescore_ctas =
      n_items > 0 ? (int)std::min<int64_t>(
                        (units + kRescoreWarps - 1) / kRescoreWarps,
                        (int64_t)sm_count * 8)
                  : sm_count * 8;
  const RescoreFn rescore = rescore_for(t.Dp);
  if (!rescore) return cudaErrorInvalidValue;
  const size_t smem = screen_smem(sd.kh);
  cudaError_t e = cudaMemsetAsync(&ctr->screen_next, 0,
                                  2 * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
#define BKD_SCREEN_KH(KH)                                                    \
  tc_prep_kernel<KH><<<aux, 128, 0, s>>>(t, sd, items, ctr, act, qpad, lst_d,   \
                                      K, w.bop);                             \
  tc_screen_kernel<KH><<<grid, kThreads, smem, s>>>(t, sd, items, 0, n_items,   \
                                                 ctr, w.bop, w.seg,          \
                                                 w.seg_cnt);
  switch (sd.kh) {
    case 1: BKD_SCREEN_KH(1) break;
    case 2: BKD_SCREEN_KH(2) break;
    case 3: BKD_SCREEN_KH(3) break;
    default: return cudaErrorInvalidValue;
  }
#undef BKD_SCREEN_KH
  rescore<<<rescore_ctas, 32 * kRescoreWarps, 0, s>>>(
      t, items, ctr, act, qpad, lst_d, lst_i, K, w.seg, w.seg_cnt, w.ovf);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // items whose survivors overflowed their segment: the float32 kernel
  return launch_leaf(t, cap, w.ovf, 0, -1, ctr, t.pts, 0, act, qpad, lst_d,
                     lst_i, K, leaf_grid, s, &ctr->screen_ovf_items);
}

}  // namespace bkd

// Test support (declared in bkd.h): the screen's MMA path on given operands.
extern "C" int bkd_probe_umma(int n, int kh, int count, const uint16_t* A,
                              const uint16_t* Bt, float* D) {
  using namespace bkd;
  set_error(BKD_OK, "");
  if (kh < 1 || kh > 3 || n < 16 || n > 256 || n % 16 != 0)
    return set_error(BKD_EINVAL, "n must be 16..256 (multiple of 16), kh 1..3");
  if (count < 0 || count > (1 << 16))
    return set_error(BKD_EINVAL, "count out of range");
  if (count == 0) return BKD_OK;
  if (!A || !Bt || !D) return set_error(BKD_EINVAL, "NULL argument");
  const size_t na = (size_t)count * 128 * 16 * kh * 2,
               nb = (size_t)count * n * 16 * kh * 2,
               nd = (size_t)count * 128 * n * 4;
  char* buf = nullptr;
  cudaError_t e = dev_malloc(&buf, na + nb + nd + sizeof(Counters));
  if (e != cudaSuccess)
    return set_error(BKD_ENOMEM, "probe buffers: %s", cudaGetErrorString(e));
  uint16_t* dA = reinterpret_cast<uint16_t*>(buf);
  uint16_t* dB = reinterpret_cast<uint16_t*>(buf + na);
  float* dD = reinterpret_cast<float*>(buf + na + nb);
  Counters* dC = reinterpret_cast<Counters*>(buf + na + nb + nd);
  int rc = BKD_OK;
  // at most two probe CTAs per SM: their tensor-memory allocations (256
  // columns each) never wait for one another
  const size_t smem = std::max<size_t>(3 * tile_bytes(kh) + 64, 100 * 1024);
  const void* kern = kh == 1   ? (const void*)umma_probe_kernel<1>
                     : kh == 2 ? (const void*)umma_probe_kernel<2>
                               : (const void*)umma_probe_kernel<3>;
  if (cudaMemcpy(dA, A, na, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dB, Bt, nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(dC, 0, sizeof(Counters)) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    rc = set_error(BKD_ECUDA, "probe set-up failed");
  } else {
    if (kh == 1)
      umma_probe_kernel<1><<<count, 128, smem>>>(n, dA, dB, dD, dC);
    else if (kh == 2)
      umma_probe_kernel<2><<<count, 128, smem>>>(n, dA, dB, dD, dC);
    else
      umma_probe_kernel<3><<<count, 128, smem>>>(n, dA, dB, dD, dC);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    Counters h{};
    if (e == cudaSuccess)
      e = cudaMemcpy(&h, dC, sizeof(Counters), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, nd, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
      rc = set_error(BKD_ECUDA, "probe failed: %s", cudaGetErrorString(e));
    else if (h.err & kErrTimeout)
      rc = set_error(BKD_ETIMEOUT, "probe MMA did not complete");
  }
  cudaFree(buf);
  return rc;
}
