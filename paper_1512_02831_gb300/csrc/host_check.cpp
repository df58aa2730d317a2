// host_check.cpp -- test support without a GPU: the host half of bkd_build
// (the median-split tree of Sec. 2.3, the node bounding boxes, and the BF16
// warp screen's operands and per-leaf bounds) into caller buffers, through
// the same functions bkd_build calls, so that CPU tests can check them
// against the oracle's tree and against exact arithmetic.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "bkd.h"
#include "bkd_internal.h"

using namespace bkd;

extern "C" int bkd_test_host_screen(const float* P, int64_t n, int d,
                                    int height, int64_t* shape,
                                    float* split, int64_t* leaf_lo,
                                    int64_t* perm,
                                    float* box, uint32_t* words,
                                    float* center, float* bmax,
                                    float* pnmax, uint16_t* tc_words) {
  if (!P || !shape) return set_error(BKD_EINVAL, "P / shape is NULL");
  if (n < 1) return set_error(BKD_EINVAL, "n must be >= 1");
  if (d < 1 || d > BKD_MAX_DIM)
    return set_error(BKD_EINVAL, "d must be in [1, %d]", BKD_MAX_DIM);
  if (height < 0 || height > BKD_MAX_HEIGHT)
    return set_error(BKD_EINVAL, "height must be in [0, %d]", BKD_MAX_HEIGHT);
  if (((int64_t)1 << height) > n)
    return set_error(BKD_EINVAL, "2^height leaves exceed n");
  for (int64_t i = 0; i < n * d; ++i)
    if (!(std::fabs(P[i]) < 1.152921504606846976e18f))
      return set_error(BKD_EINVAL, "P holds a non-finite or |x| >= 2^60 value");
  HostTree H;
  if (const char* msg = build_host_tree(P, n, d, height, &H)) {
    delete[] H.split;
    delete[] H.leaf_lo;
    delete[] H.perm;
    return set_error(BKD_ENOMEM, "%s", msg);
  }
  const int64_t L = (int64_t)1 << height;
  const int kh = screen_halves_warp(d);
  const int64_t stride = screen_stride(H.lcap);
  shape[0] = H.lcap;
  shape[1] = stride;
  shape[2] = kh;
  shape[3] = L * kh * stride * 8;  // uint32 words of the screen operands
  shape[4] = H.Dp;
  const int tkh = screen_halves(d);
  const int64_t tiles = screen_tiles(H.lcap);
  shape[5] = tiles;
  shape[6] = tkh;
  shape[7] = L * tiles * kScreenRows * 16 * tkh;  // bf16 of the tcgen05 tiles
  int rc = BKD_OK;
  if (split && leaf_lo && perm && box && words && center && bmax && pnmax &&
      tc_words) {
    std::memcpy(split, H.split, sizeof(float) * (L > 1 ? L - 1 : 1));
    std::memcpy(leaf_lo, H.leaf_lo, sizeof(int64_t) * (L + 1));
    std::memcpy(perm, H.perm, sizeof(int64_t) * n);
    fill_boxes(P, H, box);
    fill_screen_warp(P, H, stride, words, center, bmax, pnmax);
    // the tcgen05 kernel's tiles; its centre and bounds must be the same
    std::vector<float> c2((size_t)L * d), b2(L), p2(L);
    fill_screen(P, H, tiles, tc_words, c2.data(), b2.data(), p2.data());
    if (std::memcmp(c2.data(), center, sizeof(float) * L * d) != 0 ||
        std::memcmp(b2.data(), bmax, sizeof(float) * L) != 0 ||
        std::memcmp(p2.data(), pnmax, sizeof(float) * L) != 0)
      rc = set_error(BKD_EINVAL, "the two screen layouts disagree on the "
                                 "per-leaf constants");
  } else if (split || leaf_lo || perm || box || words || center || bmax ||
             pnmax || tc_words) {
    rc = set_error(BKD_EINVAL, "pass every output buffer, or none");
  }
  delete[] H.split;
  delete[] H.leaf_lo;
  delete[] H.perm;
  return rc;
}
