// k_leaf.cu -- dispatch of the leaf kernel over compiled (dimension, list
// capacity) pairs, and its launch geometry.
#include <algorithm>

#include "k_leaf.cuh"

namespace bkd {
namespace {

const void* kernel_for(int Dp, int cap) {
  switch (cap) {
    case 2: return leaf_kernel_c2(Dp);
    case 4: return leaf_kernel_c4(Dp);
    case 8: return leaf_kernel_c8(Dp);
    case 12: return leaf_kernel_c12(Dp);
    case 16: return leaf_kernel_c16(Dp);
    case 32: return leaf_kernel_c32(Dp);
    case 64: return leaf_kernel_c64(Dp);
    default: return nullptr;
  }
}

}  // namespace

int leaf_kernel_grid(int Dp, int cap, int sm_count) {
  const void* k = kernel_for(Dp, cap);
  if (!k) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kPipeThreads,
                                                    0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * sm_count;
}

cudaError_t launch_leaf(const DevTree& t, int cap, const Item* items,
                        int item_lo, int item_hi, Counters* ctr,
                        const float* pts, int64_t leaf0, const uint32_t* act,
                        const float* qpad, float* lst_d, uint32_t* lst_i,
                        int K, int grid, cudaStream_t s,
                        const int32_t* count_dev, LeafPart part) {
  if (grid <= 0) return cudaSuccess;
#define BKD_ARGS                                                          \
  t.Dp, items, item_lo, item_hi, ctr, pts, leaf0, t.leaf_cnt, t.lcap, act, \
      qpad, lst_d, lst_i, K, grid, s, count_dev, part
  switch (cap) {
    case 2: return leaf_launch_c2(BKD_ARGS);
    case 4: return leaf_launch_c4(BKD_ARGS);
    case 8: return leaf_launch_c8(BKD_ARGS);
    case 12: return leaf_launch_c12(BKD_ARGS);
    case 16: return leaf_launch_c16(BKD_ARGS);
    case 32: return leaf_launch_c32(BKD_ARGS);
    case 64: return leaf_launch_c64(BKD_ARGS);
    default: return cudaErrorInvalidValue;
  }
#undef BKD_ARGS
}

}  // namespace bkd
