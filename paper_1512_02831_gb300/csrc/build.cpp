// build.cpp -- host construction of the buffer k-d tree (Sec. 2.3, Sec. 3.1).
//
// The node at level i splits its points at the median of dimension i mod d
// (Sec. 2.3).  For a node over leaf-structure positions [lo, hi) the
// floor((hi-lo)/2) points smallest by the key (x_s, original index) go to
// [lo, mid), mid = lo + floor((hi-lo)/2); the split value is the smallest
// x_s of the right half.  Splitting stops after h levels, giving 2^h leaves
// whose sizes differ by at most one.  Sec. 3.1 builds the top tree on the
// host with linear-time selection; std::nth_element (introselect) is used per
// node, so one level costs O(n) and the whole build O(h n).
//
// Each level gathers the node-local keys (x_s, index) into a contiguous array
// (one pass over the points in their current order), selects the median of
// every node in parallel, and keeps the new order for the next level.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "bkd_internal.h"

namespace bkd {
namespace {

struct Key {
  float x;
  int32_t pad;
  int64_t idx;
};

inline bool key_less(const Key& a, const Key& b) {
  return a.x < b.x || (a.x == b.x && a.idx < b.idx);
}

int worker_count() {
  unsigned t = std::thread::hardware_concurrency();
  if (t == 0) t = 4;
  return (int)std::min(t, 64u);
}

// Runs f(lo, hi) over [0, n) split into contiguous ranges, one per worker.
template <class F>
void parallel_ranges(int64_t n, F f) {
  const int w = worker_count();
  if (n < (1 << 16) || w == 1) {
    f((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  for (int i = 0; i < w; ++i) {
    int64_t lo = n * i / w, hi = n * (i + 1) / w;
    th.emplace_back([=] { f(lo, hi); });
  }
  for (auto& t : th) t.join();
}

// Runs g(j) for j in [0, count), items handed out dynamically.
template <class G>
void parallel_items(int64_t count, G g) {
  const int w = (int)std::min<int64_t>(worker_count(), count);
  if (w <= 1) {
    for (int64_t j = 0; j < count; ++j) g(j);
    return;
  }
  std::atomic<int64_t> next{0};
  std::vector<std::thread> th;
  for (int i = 0; i < w; ++i)
    th.emplace_back([&] {
      for (int64_t j; (j = next.fetch_add(1)) < count;) g(j);
    });
  for (auto& t : th) t.join();
}

}  // namespace

int padded_dim(int d) {
  for (int D : kDims)
    if (D >= d) return D;
  return 0;
}

int list_capacity(int K) {
  for (int c : kCaps)
    if (c >= K) return c;
  return 0;
}

const char* build_host_tree(const float* P, int64_t n, int d, int h,
                            HostTree* out) {
  const int64_t L = (int64_t)1 << h;
  out->n = n;
  out->d = d;
  out->h = h;
  out->Dp = padded_dim(d);
  try {
    out->split = new float[std::max<int64_t>(L - 1, 1)];
    out->leaf_lo = new int64_t[L + 1];
    out->perm = new int64_t[n];
  } catch (...) {
    return "host allocation failed (tree arrays)";
  }
  out->split[0] = 0.f;
  std::vector<Key> keys;
  std::vector<int64_t> bounds, nb;
  try {
    keys.resize(h > 0 ? n : 0);
    bounds.reserve(L + 1);
    nb.reserve(L + 1);
  } catch (...) {
    return "host allocation failed (build keys)";
  }
  int64_t* ord = out->perm;
  parallel_ranges(n, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) ord[i] = i;
  });
  bounds.assign({0, n});
  for (int level = 0; level < h; ++level) {
    const int s = level % d;
    parallel_ranges(n, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        keys[i].x = P[ord[i] * d + s];
        keys[i].pad = 0;
        keys[i].idx = ord[i];
      }
    });
    const int64_t nodes = (int64_t)1 << level;
    nb.assign(2 * nodes + 1, 0);
    parallel_items(nodes, [&](int64_t j) {
      const int64_t lo = bounds[j], hi = bounds[j + 1];
      const int64_t mid = lo + (hi - lo) / 2;
      std::nth_element(keys.begin() + lo, keys.begin() + mid,
                       keys.begin() + hi, key_less);
      out->split[(nodes - 1) + j] = keys[mid].x;
      nb[2 * j] = lo;
      nb[2 * j + 1] = mid;
    });
    nb[2 * nodes] = n;
    parallel_ranges(n, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) ord[i] = keys[i].idx;
    });
    bounds.swap(nb);
  }
  int64_t maxleaf = 0;
  for (int64_t l = 0; l <= L; ++l) out->leaf_lo[l] = bounds[l];
  for (int64_t l = 0; l < L; ++l)
    maxleaf = std::max(maxleaf, bounds[l + 1] - bounds[l]);
  out->lcap = (maxleaf + 3) / 4 * 4;
  return nullptr;
}

void fill_quads(const float* P, const HostTree& t, int64_t leaf_a,
                int64_t leaf_b, float* pts, int64_t* orig) {
  const int d = t.d, Dp = t.Dp;
  const int64_t lcap = t.lcap;
  const float inf = INFINITY;
  parallel_items(leaf_b - leaf_a, [&](int64_t j) {
    const int64_t leaf = leaf_a + j;
    const int64_t lo = t.leaf_lo[leaf], cnt = t.leaf_lo[leaf + 1] - lo;
    for (int64_t u = 0; u < lcap; ++u) {
      const int64_t slot = j * lcap + u;  // relative to leaf_a's first slot
      float* quad = pts + (slot >> 2) * 4 * Dp;
      const int lane = (int)(slot & 3);
      if (u < cnt) {
        const int64_t row = t.perm[lo + u];
        const float* x = P + row * d;
        for (int i = 0; i < Dp; ++i) quad[4 * i + lane] = i < d ? x[i] : 0.f;
        orig[slot] = row;
      } else {
        for (int i = 0; i < Dp; ++i) quad[4 * i + lane] = inf;
        orig[slot] = -1;
      }
    }
  });
}

void fill_boxes(const float* P, const HostTree& t, float* box) {
  const int d = t.d, Dp = t.Dp;
  const int64_t L = (int64_t)1 << t.h;
  const int64_t first_leaf = L - 1;
  parallel_items(L, [&](int64_t leaf) {
    float* lo = box + (first_leaf + leaf) * 2 * Dp;
    float* hi = lo + Dp;
    for (int i = 0; i < Dp; ++i) {
      // padding dimensions: q_i = 0 lies in [0, 0] and adds nothing
      lo[i] = i < d ? INFINITY : 0.f;
      hi[i] = i < d ? -INFINITY : 0.f;
    }
    for (int64_t p = t.leaf_lo[leaf]; p < t.leaf_lo[leaf + 1]; ++p) {
      const float* x = P + t.perm[p] * d;
      for (int i = 0; i < d; ++i) {
        lo[i] = std::min(lo[i], x[i]);
        hi[i] = std::max(hi[i], x[i]);
      }
    }
  });
  for (int64_t v = first_leaf - 1; v >= 0; --v) {
    float* b = box + v * 2 * Dp;
    const float* l = box + (2 * v + 1) * 2 * Dp;
    const float* r = box + (2 * v + 2) * 2 * Dp;
    for (int i = 0; i < Dp; ++i) {
      b[i] = std::min(l[i], r[i]);
      b[Dp + i] = std::max(l[Dp + i], r[Dp + i]);
    }
  }
}

namespace {

// Floor of a leaf's pn_max.  The screens' error term E holds 2^-14 pn_max,
// so E >= 2^-100: the absolute errors that underflow adds (products or an
// accumulator below 2^-126, the norm split of a subnormal pn, |v_hat|^2
// below 2^-126) stay under 2^-118 and are covered; for any leaf whose
// points are not all within ~2^-43 of its centre the floor changes nothing.
constexpr float kPnMaxFloor = 0x1p-86f;

// float -> bfloat16, round to nearest even (inputs are finite).
inline uint16_t bf16_rn(float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  const uint32_t lsb = (x >> 16) & 1u;
  return (uint16_t)((x + 0x7fffu + lsb) >> 16);
}

inline float bf16_to_float(uint16_t h) {
  const uint32_t x = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &x, 4);
  return f;
}

}  // namespace

namespace {

// One leaf of either screen layout: its centre c (midpoint of the leaf's
// bounding box) into `c`, then `rows` rows of bf16 slots -- the point's
// offsets bf16(fl(x - c)) in 0..d-1 and its squared norm pn (binary64 sum
// rounded to float) split as pn_hi = bf16(pn), pn_lo = bf16(pn - pn_hi) in
// d, d+1; rows past the leaf's points hold pn_hi = +inf and zeros -- each
// handed to place(u, hv, real); finally the leaf's bmax and pnmax.
template <class Place>
void screen_leaf(const float* P, const HostTree& t, int64_t leaf,
                 int64_t rows, float* c, float* bmax, float* pnmax,
                 Place place) {
  const int d = t.d;
  // BF16 rounding error (relative, round to nearest: 8 significant bits, so
  // 2^-8) with margin for the float32 subtraction before it, and its effect
  // on a norm: |w_hat - w| <= rho |w|, |w| <= |w_hat| / (1 - rho).
  const double rho = std::ldexp(1.0, -8) * (1.0 + 1e-4);
  const double tiny = std::ldexp(1.0, -126) * std::sqrt((double)d);
  const int64_t lo = t.leaf_lo[leaf], cnt = t.leaf_lo[leaf + 1] - lo;
  for (int i = 0; i < d; ++i) {
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t u = 0; u < cnt; ++u) {
      const float x = P[t.perm[lo + u] * d + i];
      mn = std::min(mn, x);
      mx = std::max(mx, x);
    }
    c[i] = 0.5f * mn + 0.5f * mx;
  }
  double wmax = 0.0;
  float pmax = 0.f;
  for (int64_t u = 0; u < rows; ++u) {
    uint16_t hv[48] = {0};
    const bool real = u < cnt;
    if (real) {
      const float* x = P + t.perm[lo + u] * d;
      double ss = 0.0;
      for (int i = 0; i < d; ++i) {
        hv[i] = bf16_rn(x[i] - c[i]);
        const double w = bf16_to_float(hv[i]);
        ss += w * w;
      }
      const float pv = (float)ss;
      // pv - pn_hi is exact (at most 16 significant bits remain); its
      // bf16 rounding leaves pn_hi + pn_lo within 2^-16 pv of pv
      hv[d] = bf16_rn(pv);
      hv[d + 1] = bf16_rn(pv - bf16_to_float(hv[d]));
      wmax = std::max(wmax, std::sqrt(ss));
      pmax = std::max(pmax, pv);
    } else {
      hv[d] = 0x7f80;  // +inf: the row's product is -inf, never kept
    }
    place(u, hv, real);
  }
  *bmax = std::nextafter((float)(rho / (1.0 - rho) * wmax + tiny), INFINITY);
  *pnmax = std::nextafter(std::max(pmax, kPnMaxFloor), INFINITY);
}

}  // namespace

void fill_screen(const float* P, const HostTree& t, int64_t tiles,
                 uint16_t* words, float* center, float* bmax, float* pnmax) {
  const int d = t.d;
  const int kh = screen_halves(d);
  const int64_t L = (int64_t)1 << t.h;
  const int64_t tile_elems = (int64_t)kScreenRows * 16 * kh;  // bf16 per tile
  const uint16_t one = 0x3f80;  // bf16 1.0
  parallel_items(L, [&](int64_t leaf) {
    uint16_t* lw = words + leaf * tiles * tile_elems;
    screen_leaf(P, t, leaf, tiles * kScreenRows, center + leaf * d,
                bmax + leaf, pnmax + leaf,
                [&](int64_t u, uint16_t* hv, bool real) {
                  // the three threshold slots of the query column meet 1.0
                  if (real) hv[d + 2] = hv[d + 3] = hv[d + 4] = one;
                  // tile T = u / 128, row r = u % 128; the row's 2 kh groups
                  // of eight slots go to the canonical no-swizzle K-major
                  // layout of the MMA operand (screen_row_offset)
                  uint16_t* tile = lw + (u / kScreenRows) * tile_elems;
                  const int r = (int)(u % kScreenRows);
                  for (int kg = 0; kg < 2 * kh; ++kg)
                    for (int e = 0; e < 8; ++e)
                      tile[screen_row_offset(r, kg, kh) / 2 + e] =
                          hv[8 * kg + e];
                });
  });
}

void fill_screen_warp(const float* P, const HostTree& t, int64_t stride,
                      uint32_t* words, float* center, float* bmax,
                      float* pnmax) {
  const int d = t.d;
  const int kh = screen_halves_warp(d);
  const int64_t L = (int64_t)1 << t.h;
  parallel_items(L, [&](int64_t leaf) {
    screen_leaf(
        P, t, leaf, stride, center + leaf * d, bmax + leaf, pnmax + leaf,
        [&](int64_t u, const uint16_t* hv, bool) {
          // 32-point super-tiles S = u / 32 of two 16-point m-tiles a; in
          // tile a the point is row 8 r + g (r = 0, 1; g = 0..7).  Lane
          // (g, t) of a warp loads, with one 16-byte load per row half r,
          // words (t, t + 4) of row 8 r + g of both tiles: its m16n8k16 A
          // fragments.
          const int64_t S = u / 32, a = (u % 32) / 16, r = (u % 16) / 8,
                        g = u % 8;
          for (int h = 0; h < kh; ++h) {
            // word j of a k-half = slots (2j, 2j+1) of the half
            uint32_t* blk = words + (leaf * kh + h) * stride * 8 +
                            ((S * 2 + r) * 8 + g) * 16 + 2 * a;
            for (int tq = 0; tq < 4; ++tq)
              for (int e = 0; e < 2; ++e) {
                const int k0 = 16 * h + 2 * (tq + 4 * e);
                blk[tq * 4 + e] =
                    (uint32_t)hv[k0] | ((uint32_t)hv[k0 + 1] << 16);
              }
          }
        });
  });
}

}  // namespace bkd
