// traverse.cuh -- one step of a query's implicit tree traversal (Sec. 2.3,
// Sec. 2.4): from the leaf visited last to the next leaf the search must
// visit, or kDone once the traversal has reached the root twice.
//
// Order: the depth-first order of the classical search -- near child (the
// side of the split that holds q) before far child.  Stackless: the state is
// the heap index of the last leaf.  The path from the root to it is encoded
// in the index bits, so a pass over the path recovers every ancestor whose
// far child is still unvisited (the path went through its near child) -- the
// recursive search's backtracking stack -- and the next subtree to enter is
// the far child of the DEEPEST such ancestor that survives pruning.
//
// Pruning: a subtree is skipped when the distance from q to the bounding box
// of its points cannot beat the query's current bound.  This refines the
// paper's hyperplane test (the box lies beyond the hyperplane, so its
// distance is never smaller) and changes only how many leaves are visited,
// never the result:
//   * float32 pass: per dimension o_i = fl(lo_i - q_i) or fl(q_i - hi_i)
//     (0 inside the box) and B = fl(o_0^2), B = fma(o_i, o_i, B) for
//     i = 1..d-1 -- the same float32 chain that scores a point.  For every
//     point x in the box |fl(q_i - x_i)| >= o_i (rounding is monotone) and
//     each chain step is monotone in both arguments, so B <= the float32
//     distance of every point below the node.  A point enters a list only if
//     its distance is strictly below the list's last entry `bound`, so
//     skipping when B >= bound is exact.
//   * binary64 search: o_i in binary64 (exact differences of floats) and
//     B = sum of o_i^2 in dimension order from 0.0 -- the oracle's sequence --
//     so B <= the binary64 distance of every point below; points enter on the
//     key (D, index), so a subtree is visited while B <= bound.
// A subtree whose near child is skipped is left through its last leaf in
// depth-first order (always taking the far side), which marks it visited.
#pragma once

#include "bkd_internal.h"

namespace bkd {

__device__ __forceinline__ int heap_level(int v) { return 31 - __clz(v + 1); }

// float32 pruning bound of one query; D = Dp (compile time), the query in
// registers and each box read as 2D/4 16-byte loads.  Padding dimensions
// (q_i = 0, box [0, 0]) add fma(0, 0, B) = B.
template <int D>
struct F32Bound {
  using T = float;
  float x[D];
  __device__ void load(const float* __restrict__ qp) {
#pragma unroll
    for (int i = 0; i < D; ++i) x[i] = qp[i];
  }
  __device__ static bool keep(float b, float bound) { return b < bound; }
  __device__ float box(const DevTree& t, int node) const {
    static_assert(D % 2 == 0, "a box row pair is a whole number of float4");
    const float4* p =
        reinterpret_cast<const float4*>(t.box + (size_t)node * 2 * D);
    float f[2 * D];
#pragma unroll
    for (int j = 0; j < D / 2; ++j) {
      const float4 v = __ldg(p + j);
      f[4 * j] = v.x;
      f[4 * j + 1] = v.y;
      f[4 * j + 2] = v.z;
      f[4 * j + 3] = v.w;
    }
    float b = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float q = x[i], l = f[i], u = f[D + i];
      const float o = q < l ? __fsub_rn(l, q) : (q > u ? __fsub_rn(q, u) : 0.f);
      b = i == 0 ? __fmul_rn(o, o) : __fmaf_rn(o, o, b);
    }
    return b;
  }
  __device__ static float plane(float q, float t) {
    const float g = q < t ? __fsub_rn(t, q) : __fsub_rn(q, t);
    return __fmul_rn(g, g);
  }
};

// binary64 pruning bound of one query (the oracle's sequence).
struct F64Bound {
  using T = double;
  const float* qp;
  __device__ static bool keep(double b, double bound) { return b <= bound; }
  __device__ double box(const DevTree& t, int node) const {
    const float* lo = t.box + (size_t)node * 2 * t.Dp;
    const float* hi = lo + t.Dp;
    double b = 0.0;
    for (int i = 0; i < t.d; ++i) {
      const double q = qp[i], l = __ldg(lo + i), u = __ldg(hi + i);
      const double o = q < l ? __dsub_rn(l, q) : (q > u ? __dsub_rn(q, u) : 0.0);
      b = __dadd_rn(b, __dmul_rn(o, o));
    }
    return b;
  }
  __device__ static double plane(float q, float t) {
    const double g = __dsub_rn((double)q, (double)t);
    return __dmul_rn(g, g);
  }
};

// Last leaf, in depth-first order, of the subtree of u (always the far side).
// The split dimension of level l is l mod d, stepped incrementally.
__device__ __forceinline__ int last_leaf(const DevTree& t,
                                         const float* __restrict__ qp, int u) {
  const int first_leaf = (1 << t.h) - 1;
  int dim = heap_level(u) % t.d;
  while (u < first_leaf) {
    u = 2 * u + (qp[dim] < __ldg(t.split + u) ? 2 : 1);
    dim = dim + 1 == t.d ? 0 : dim + 1;
  }
  return u;
}

// Deepest unvisited far child on the path of leaf `node` that survives
// pruning, or -1.
template <class B>
__device__ __forceinline__ int climb(const DevTree& t, const B& bx,
                                     const float* __restrict__ qp, int node,
                                     typename B::T bound) {
  const int h = t.h, d = t.d;
  if (node == 0) return -1;
  const unsigned path = (unsigned)(node + 1);
  int dim = (h - 1) % d;
  for (int level = h - 1; level >= 0;
       --level, dim = dim == 0 ? d - 1 : dim - 1) {
    const int anc = (int)(path >> (h - level)) - 1;
    const float sv = __ldg(t.split + anc);
    const float qs = qp[dim];
    const bool near_left = qs < sv;
    const bool went_left = ((path >> (h - 1 - level)) & 1u) == 0u;
    if (went_left != near_left) continue;  // far child already on the path
    if (!B::keep(B::plane(qs, sv), bound)) continue;  // box is beyond plane
    const int far = 2 * anc + (near_left ? 2 : 1);
    if (B::keep(bx.box(t, far), bound)) return far;
  }
  return -1;
}

// Next leaf (heap index) to visit after leaf `node` (kStart: enter at the
// root), or kDone.
template <class B>
__device__ __forceinline__ int next_leaf(const DevTree& t, const B& bx,
                                         const float* __restrict__ qp,
                                         int node, typename B::T bound) {
  const int first_leaf = (1 << t.h) - 1;
  int cand;
  if (node == kStart) {
    if (!B::keep(bx.box(t, 0), bound)) return kDone;
    cand = 0;
  } else {
    cand = climb<B>(t, bx, qp, node, bound);
  }
  while (cand >= 0) {
    int v = cand;
    int dim = heap_level(v) % t.d;
    while (v < first_leaf) {
      const int nc = 2 * v + (qp[dim] < __ldg(t.split + v) ? 1 : 2);
      dim = dim + 1 == t.d ? 0 : dim + 1;
      if (B::keep(bx.box(t, nc), bound)) {
        v = nc;
      } else {  // the near child holds nothing better: skip its subtree
        node = last_leaf(t, qp, nc);
        v = -1;
        break;
      }
    }
    if (v >= 0) return v;
    cand = climb<B>(t, bx, qp, node, bound);
  }
  return kDone;
}

}  // namespace bkd
