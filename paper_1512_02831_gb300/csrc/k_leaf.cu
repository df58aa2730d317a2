// k_leaf.cu -- dispatch of the leaf kernel over compiled (dimension, list
// capacity) pairs, and its launch geometry.
#include <algorithm>

#include "k_leaf.cuh"

namespace bkd {
namespace {

// Shared memory staged per CTA: one leaf segment.  48 KB keeps 4-5 CTAs of
// 128 threads resident per SM next to their registers.
constexpr int64_t kSegBytes = 48 * 1024;

int seg_quads_for(int Dp, int64_t lcap) {
  const int64_t per_quad = (int64_t)Dp * 16;
  return (int)std::max<int64_t>(1, std::min<int64_t>(lcap / 4,
                                                      kSegBytes / per_quad));
}

const void* kernel_for(int variant, int Dp, int cap) {
  switch (cap) {
    case 2: return leaf_kernel_c2(variant, Dp);
    case 4: return leaf_kernel_c4(variant, Dp);
    case 8: return leaf_kernel_c8(variant, Dp);
    case 12: return leaf_kernel_c12(variant, Dp);
    case 16: return leaf_kernel_c16(variant, Dp);
    case 32: return leaf_kernel_c32(variant, Dp);
    default: return nullptr;
  }
}

}  // namespace

int leaf_kernel_grid(int variant, int Dp, int cap, int64_t lcap,
                     int sm_count) {
  const void* k = kernel_for(variant, Dp, cap);
  if (!k) return 0;
  const bool cta = variant == kLeafCta;
  const size_t smem = cta ? (size_t)seg_quads_for(Dp, lcap) * Dp * 16 : 0;
  const int threads = cta ? kTileQ : kPipeThreads;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads,
                                                    smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * sm_count;
}

int leaf_grid_units(int variant, int n_items) {
  (void)variant;  // both kernels take one item per CTA at a time
  return n_items;
}

cudaError_t launch_leaf(int variant, int Dp, int cap, const Item* items,
                        int item_lo,
                        int item_hi, Counters* ctr, const float* pts,
                        int64_t leaf0, const int32_t* leaf_cnt, int64_t lcap,
                        const uint32_t* act, const float* qpad, float* lst_d,
                        uint32_t* lst_i, int K, int grid, cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  const int seg = seg_quads_for(Dp, lcap);
  const size_t smem = (size_t)seg * Dp * 16;
#define BKD_ARGS                                                             \
  variant, Dp, items, item_lo, item_hi, ctr, pts, leaf0, leaf_cnt, lcap, act, qpad, \
      lst_d, lst_i, K, grid, seg, smem, s
  switch (cap) {
    case 2: return leaf_launch_c2(BKD_ARGS);
    case 4: return leaf_launch_c4(BKD_ARGS);
    case 8: return leaf_launch_c8(BKD_ARGS);
    case 12: return leaf_launch_c12(BKD_ARGS);
    case 16: return leaf_launch_c16(BKD_ARGS);
    case 32: return leaf_launch_c32(BKD_ARGS);
    default: return cudaErrorInvalidValue;
  }
#undef BKD_ARGS
}

}  // namespace bkd
