// k_screen.cu -- ProcessAllBuffers with a BF16 tensor-core screen.
//
// Same work items and same result as the float32 leaf kernel (every point
// whose float32 distance could still enter a query's candidate list is scored
// exactly), but most points are rejected by a cheap screen first:
//
//   v = q - c, w = x - c (c: centre of the leaf), rounded to bf16 (v^, w^);
//   s = |v^|^2 + |w^|^2 - 2 v^.w^, the dot products on the tensor cores
//   (mma.sync m16n8k16, bf16 in, fp32 accumulate: 16 queries x 8 points per
//   instruction and 16-dimension half).
//
// Safety bound.  With rho = 2^-9 (1 + 1e-4) (bf16 round-to-nearest plus the
// float32 subtraction), |v^ - v| <= rho |v| and |v| <= |v^| / (1 - rho), so
//   |q - x| >= |v^ - w^| - A_q - B_x,  A_q = rho/(1-rho) |v^|,
// and B_x <= B_max, the leaf's largest such term (prepared on the host).  The
// computed s differs from |v^ - w^|^2 by at most E = 2^-15 (|v^|^2 + pn_max)
// (fp32 accumulation inside the tensor core at up to 2^-22 per addition over
// 16 terms, the rounding of |v^|^2, |w^|^2 and of the epilogue, with a 4x
// margin).  The float32 distance of the exact path obeys
// D32 >= D (1 - g) - eta, g = (d+3) 2^-24, eta = 2^-120.  Hence a point can
// only enter the list (D32 < bound) if
//   s < (sqrt((bound + eta) / (1 - g)) + A_q + B_max)^2 + E,
// evaluated once per (query, leaf) in float32 with every operation rounded
// toward the larger threshold (divisors toward the smaller).  Kept
// points are scored with the exact float32 chain of the leaf kernel and
// inserted with the same strict rule, so the lists -- and the answers -- are
// bit for bit those of the float32 path.
#include <cuda_bf16.h>

#include "bkd.h"
#include "bkd_internal.h"
#include "k_leaf.cuh"

namespace bkd {
namespace {

constexpr int kScrWarps = 4;  // 4 warps x 16 queries = one 64-query item
constexpr int kScrThreads = kScrWarps * 32;
static_assert(kScrWarps * 16 == kPipeTile, "screen item = leaf item");

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

// d[0..3] = a (16x16 bf16, row) x b (16x8 bf16, col) + c, fp32.
__device__ __forceinline__ void mma_bf16(float (&acc)[4], const uint32_t (&a)[4],
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
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

struct ScreenArgs {
  const uint32_t* words;  // packed bf16 offsets, see fill_screen
  const float* pn;        // |w^|^2 per slot
  const float* center;    // d floats per leaf
  const float* bmax;      // per leaf
  const float* pnmax;     // per leaf
  int kh;                 // 16-dimension halves
};

// Per-warp setup of the warp's 16 query rows of item w: query ids, the
// candidate lists (copied into shared memory), the bf16 offsets (A operand
// record) and the screen thresholds.  Lanes 0..15, row = 16 * warp + lane.
template <int KH>
__device__ __forceinline__ void setup_rows(
    const DevTree& t, const ScreenArgs& sc, const Item& w, int warp, int lane,
    const uint32_t* __restrict__ act, const float* __restrict__ qpad,
    const float* __restrict__ lst_d, const uint32_t* __restrict__ lst_i,
    int K, float* s_ld, uint32_t* s_li, uint32_t* s_rows, float* s_thr,
    uint32_t* s_q) {
  if (lane >= 16) return;
  const float inf = __int_as_float(0x7f800000);
  const int r = warp * 16 + lane;
  uint32_t* rec = s_rows + (size_t)warp * KH * 16 * 8;
  float thr = -inf;  // empty rows keep nothing
  if (r < w.count) {
    const uint32_t q = act[w.start + r];
    s_q[r] = q;
    for (int j = 0; j < K; ++j) {
      s_ld[r * K + j] = lst_d[(size_t)q * K + j];
      s_li[r * K + j] = lst_i[(size_t)q * K + j];
    }
    const float* qp = qpad + (size_t)q * t.Dp;
    const float* c = sc.center + (size_t)w.leaf * t.d;
    float qn = 0.f, ss = 0.f;  // |v^|^2 rounded to nearest / upward
    for (int h = 0; h < KH; ++h)
      for (int j = 0; j < 8; ++j) {
        const int k0 = 16 * h + 2 * j;
        const float a0 = k0 < t.d ? __fsub_rn(qp[k0], c[k0]) : 0.f;
        const float a1 = k0 + 1 < t.d ? __fsub_rn(qp[k0 + 1], c[k0 + 1]) : 0.f;
        const uint32_t wd = pack_bf16(a0, a1);
        rec[(h * 16 + lane) * 8 + (j < 4 ? 2 * j : 2 * (j - 4) + 1)] = wd;
        const float v0 = bf16_lo(wd), v1 = bf16_hi(wd);
        qn = __fmaf_rn(v0, v0, qn);
        qn = __fmaf_rn(v1, v1, qn);
        ss = __fmaf_ru(v0, v0, ss);
        ss = __fmaf_ru(v1, v1, ss);
      }
    const float bound = s_ld[r * K + K - 1];
    if (isinf(bound)) {
      thr = inf;
    } else {
      // the bound of the header comment, every step rounded upward
      // (divisors downward) so the float result is never too small
      const float rho = 0x1p-9f * 1.0001f;
      const float rr = __fdiv_ru(rho, __fsub_rd(1.f, rho));
      const float one_m_g = __fsub_rd(1.f, (float)(t.d + 3) * 0x1p-24f);
      const float aq = __fadd_ru(__fmul_ru(rr, __fsqrt_ru(ss)), 0x1p-123f);
      const float R =
          __fsqrt_ru(__fdiv_ru(__fadd_ru(bound, 0x1p-120f), one_m_g));
      const float Rb = __fadd_ru(__fadd_ru(R, aq), sc.bmax[w.leaf]);
      const float E = __fmul_ru(0x1p-15f, __fadd_ru(ss, sc.pnmax[w.leaf]));
      thr = __fsub_ru(__fadd_ru(__fmul_ru(Rb, Rb), E), qn);
    }
  } else {
    for (int h = 0; h < KH; ++h)
      for (int j = 0; j < 8; ++j) rec[(h * 16 + lane) * 8 + j] = 0u;
  }
  s_thr[r] = thr;
}

// Shared memory of one CTA (lcap8 = slots per leaf rounded up to 8):
//   words  KH * lcap8 * 8 u32   the leaf's packed bf16 offsets
//   pn     lcap8 f32            their squared norms (+inf past the leaf)
//   ld, li 64 * K f32 / u32     the item's candidate lists
//   rows   4 * KH * 16 * 8 u32  each warp's 16 query offsets (A operand)
//   thr    64 f32               screen thresholds (minus |v^|^2)
//   qid    64 u32               query ids
// A CTA takes a contiguous range of items; consecutive items of the same
// leaf reuse the staged leaf, a new leaf arrives by two TMA bulk copies
// (offsets, norms) on one mbarrier while the warps set up their rows.
template <int KH>
__global__ void __launch_bounds__(kScrThreads)
    screen_kernel(DevTree t, ScreenArgs sc, const Item* __restrict__ items,
                  int item_lo, int item_hi, Counters* ctr,
                  const uint32_t* __restrict__ act,
                  const float* __restrict__ qpad, float* __restrict__ lst_d,
                  uint32_t* __restrict__ lst_i, int K, int lcap8) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t full;
  uint32_t* s_words = reinterpret_cast<uint32_t*>(smem);
  float* s_pn = reinterpret_cast<float*>(s_words + (size_t)KH * lcap8 * 8);
  float* s_ld = s_pn + lcap8;
  uint32_t* s_li = reinterpret_cast<uint32_t*>(s_ld + 64 * K);
  uint32_t* s_rows = s_li + 64 * K;
  float* s_thr = reinterpret_cast<float*>(s_rows + kScrWarps * KH * 16 * 8);
  uint32_t* s_q = reinterpret_cast<uint32_t*>(s_thr + 64);
  const float inf = __int_as_float(0x7f800000);
  const int hi = item_hi >= 0 ? item_hi : ctr->n_items;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const unsigned full_mask = 0xffffffffu;
  const int lcap = (int)t.lcap;
  const uint32_t bar = smem_u32(&full);
  // slots past the leaf: zero offsets, +inf norms (never kept)
  for (int h = 0; h < KH; ++h)
    for (int i = lcap * 8 + tid; i < lcap8 * 8; i += kScrThreads)
      s_words[(size_t)h * lcap8 * 8 + i] = 0u;
  for (int i = lcap + tid; i < lcap8; i += kScrThreads) s_pn[i] = inf;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const int n = hi - item_lo;
  const int per = (n + (int)gridDim.x - 1) / (int)gridDim.x;
  const int it0 = item_lo + (int)blockIdx.x * per;
  const int it1 = min(hi, it0 + per);
  int staged = -1;
  uint32_t parity = 0;
  unsigned long long kept = 0;
  for (int it = it0; it < it1; ++it) {
    const Item w = items[it];
    const bool fresh = w.leaf != staged;
    if (fresh) {
      __syncthreads();  // every warp is done with the previous leaf
      if (tid == 0) {
        async_proxy_fence();
        const uint32_t wbytes = (uint32_t)lcap * 32u;
        const uint32_t pbytes = (uint32_t)lcap * 4u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::
                         "r"(bar),
                     "r"((uint32_t)KH * wbytes + pbytes)
                     : "memory");
        for (int h = 0; h < KH; ++h)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::"
              "bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_u32(s_words + (size_t)h * lcap8 * 8)),
              "l"(__cvta_generic_to_global(
                  sc.words + (((size_t)w.leaf * KH + h) * lcap) * 8)),
              "r"(wbytes), "r"(bar)
              : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::"
            "bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(s_pn)),
            "l"(__cvta_generic_to_global(sc.pn + (size_t)w.leaf * lcap)),
            "r"(pbytes), "r"(bar)
            : "memory");
      }
      staged = w.leaf;
    }
    setup_rows<KH>(t, sc, w, warp, lane, act, qpad, lst_d, lst_i, K, s_ld,
                   s_li, s_rows, s_thr, s_q);
    __syncwarp();
    if (fresh) {
      const bool ok = mbar_wait(bar, parity);
      parity ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicOr(&ctr->err, kErrTimeout);
          mbar_wait(bar, parity ^ 1u);  // bounded: let the copy land
        }
        return;
      }
    }
    const int npt = t.leaf_cnt[w.leaf];
    const int ntile = (npt + 7) >> 3;
    const int wr0 = warp * 16;
    if (wr0 < w.count) {  // warp-uniform
      uint32_t a[KH][4];
      const uint32_t* rb = s_rows + (size_t)warp * KH * 16 * 8;
#pragma unroll
      for (int h = 0; h < KH; ++h) {
        const uint2 x0 =
            *reinterpret_cast<const uint2*>(rb + (h * 16 + g) * 8 + 2 * tq);
        const uint2 x1 =
            *reinterpret_cast<const uint2*>(rb + (h * 16 + g + 8) * 8 + 2 * tq);
        a[h][0] = x0.x;
        a[h][1] = x1.x;
        a[h][2] = x0.y;
        a[h][3] = x1.y;
      }
      const float thr_g = s_thr[wr0 + g], thr_g8 = s_thr[wr0 + g + 8];
      for (int nt = 0; nt < ntile; ++nt) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int h = 0; h < KH; ++h) {
          const uint2 b = *reinterpret_cast<const uint2*>(
              s_words + ((size_t)h * lcap8 + nt * 8 + g) * 8 + 2 * tq);
          mma_bf16(acc, a[h], b.x, b.y);
        }
        const float2 p2 = *reinterpret_cast<const float2*>(s_pn + nt * 8 + 2 * tq);
        float y[4];
        y[0] = __fmaf_rn(-2.f, acc[0], p2.x);
        y[1] = __fmaf_rn(-2.f, acc[1], p2.y);
        y[2] = __fmaf_rn(-2.f, acc[2], p2.x);
        y[3] = __fmaf_rn(-2.f, acc[3], p2.y);
        const bool keep =
            fminf(y[0], y[1]) < thr_g || fminf(y[2], y[3]) < thr_g8;
        if (__any_sync(full_mask, keep)) {
          // exact rescoring; the four lanes of a group share rows g and
          // g + 8, so they take turns
          for (int turn = 0; turn < 4; ++turn) {
            if (tq == turn && keep) {
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int row = wr0 + g + 8 * (j >> 1);
                const int col = nt * 8 + 2 * tq + (j & 1);
                if (y[j] < (j < 2 ? thr_g : thr_g8) && col < npt) {
                  ++kept;
                  const uint32_t slot =
                      (uint32_t)((int64_t)w.leaf * t.lcap + col);
                  const float dv = exact_dist(qpad + (size_t)s_q[row] * t.Dp,
                                              t.pts, t.Dp, slot);
                  float* ld = s_ld + row * K;
                  uint32_t* li = s_li + row * K;
                  if (dv < ld[K - 1]) {
                    int pos = K - 1;
                    while (pos > 0 && ld[pos - 1] > dv) {
                      ld[pos] = ld[pos - 1];
                      li[pos] = li[pos - 1];
                      --pos;
                    }
                    ld[pos] = dv;
                    li[pos] = slot;
                  }
                }
              }
            }
            __syncwarp();
          }
        }
      }
    }
    __syncwarp();
    if (lane < 16) {  // write the warp's rows back
      const int r = wr0 + lane;
      if (r < w.count) {
        const uint32_t q = s_q[r];
        for (int j = 0; j < K; ++j) {
          lst_d[(size_t)q * K + j] = s_ld[r * K + j];
          lst_i[(size_t)q * K + j] = s_li[r * K + j];
        }
      }
    }
    __syncwarp();
  }
  if (kept) atomicAdd(&ctr->screen_kept, kept);
}

size_t screen_smem(int kh, int lcap8, int K) {
  return (size_t)kh * lcap8 * 32 + (size_t)lcap8 * 4 + (size_t)64 * K * 8 +
         (size_t)kScrWarps * kh * 16 * 32 + 64 * 4 + 64 * 4;
}

}  // namespace

int screen_grid(int kh, int64_t lcap, int K, int sm_count) {
  const int lcap8 = (int)((lcap + 7) / 8 * 8);
  const size_t smem = screen_smem(kh, lcap8, K);
  const void* k = kh == 1 ? reinterpret_cast<const void*>(&screen_kernel<1>)
                          : reinterpret_cast<const void*>(&screen_kernel<2>);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kScrThreads,
                                                    smem) != cudaSuccess)
    return 0;
  return per_sm * sm_count;
}

cudaError_t launch_screen(const DevTree& t, const ScreenData& sd,
                          const Item* items, int item_lo, int item_hi,
                          Counters* ctr, const uint32_t* act,
                          const float* qpad, float* lst_d, uint32_t* lst_i,
                          int K, int grid, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  const int lcap8 = (int)((t.lcap + 7) / 8 * 8);
  const size_t smem = screen_smem(sd.kh, lcap8, K);
  ScreenArgs sc{sd.words, sd.pn, sd.center, sd.bmax, sd.pnmax, sd.kh};
  if (sd.kh == 1)
    screen_kernel<1><<<grid, kScrThreads, smem, s>>>(
        t, sc, items, item_lo, item_hi, ctr, act, qpad, lst_d, lst_i, K, lcap8);
  else
    screen_kernel<2><<<grid, kScrThreads, smem, s>>>(
        t, sc, items, item_lo, item_hi, ctr, act, qpad, lst_d, lst_i, K, lcap8);
  return cudaGetLastError();
}

}  // namespace bkd
