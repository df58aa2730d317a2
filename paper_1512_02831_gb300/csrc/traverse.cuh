// traverse.cuh -- one step of a query's implicit tree traversal (Sec. 2.3,
// Sec. 2.4): from the leaf visited last to the next leaf the search must
// visit, or kDone once the traversal has reached the root twice.
//
// Order: the depth-first order of the classical search -- near child (the
// side of the split that holds q) before far child.  State: the heap index
// of the last leaf (its bits encode the path from the root) and a mask with
// bit l set when the child of the level-l ancestor that is NOT on the path
// needs no further visit: the path went through the far child there (the
// near child was visited before), or the far child was pruned.  The mask is
// the recursive search's backtracking stack in 32 bits: the next subtree to
// enter is the far child at the deepest level whose bit is clear and that
// survives pruning.  A far child is tested at most once: pruned, it stays
// pruned (the bound only shrinks); entered, it is on the path.
//
// Pruning: a subtree is skipped when the distance from q to the bounding box
// of its points cannot beat the query's current bound.  This refines the
// paper's hyperplane test (the box lies beyond the hyperplane, so its
// distance is never smaller) and changes only how many leaves are visited,
// never the result:
// per dimension o_i = fl(lo_i - q_i) or fl(q_i - hi_i) (0 inside the box)
// and B = fl(o_0^2), B = fma(o_i, o_i, B) for i = 1..d-1 -- the same float32
// chain that scores a point.  For every point x in the box
// |fl(q_i - x_i)| >= o_i (rounding is monotone) and each chain step is
// monotone in both arguments, so B <= the float32 distance of every point
// below the node.  A point enters a list only if its distance is strictly
// below the list's last entry `bound`, so skipping when B >= bound is exact.
// (The binary64 fallback search passes a bound widened to cover its
// binary64 key, see k_exact.cu.)
// A near child that is pruned counts as visited: the walk continues with the
// far child of its parent.
#pragma once

#include "bkd_internal.h"

namespace bkd {

__device__ __forceinline__ int heap_level(int v) { return 31 - __clz(v + 1); }

// max(a, b, c) (three-input float max of sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

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
      // fl(l - q) if q < l, fl(q - u) if q > u, else 0 (the other
      // difference is then <= 0): one three-input max
      const float q = x[i];
      const float o = fmax3(__fsub_rn(f[i], q), __fsub_rn(q, f[D + i]), 0.f);
      b = i == 0 ? __fmul_rn(o, o) : __fmaf_rn(o, o, b);
    }
    return b;
  }
};

// Ancestor of heap node u (at level lu) at level l <= lu.
__device__ __forceinline__ int ancestor(int u, int lu, int l) {
  return (int)(((unsigned)u + 1u) >> (lu - l)) - 1;
}

// Next leaf (heap index) to visit after `node` (kStart: enter at the root),
// or kDone; `mask` (see the header) is updated to the returned leaf's path.
// One loop for both directions, one box test per iteration, so that the
// lanes of a warp -- each on its own query -- stay in step as far as their
// paths allow.  (The paper's hyperplane test needs no separate pass: the box
// of a far child lies beyond the plane, so its bound is never smaller, in
// either precision, and it prunes everything the plane test would.)
template <class B>
__device__ __forceinline__ int next_leaf(const DevTree& t, const B& bx,
                                         const float* __restrict__ qp,
                                         int node, uint32_t& mask,
                                         typename B::T bound) {
  const int h = t.h;
  int u;      // descending: the node entered last; climbing: a finished node
  bool down;  // descending (near child next) or climbing (open far child)
  if (node == kStart) {
    mask = 0u;
    if (!B::keep(bx.box(t, 0), bound)) return kDone;
    u = 0;
    down = true;
  } else {
    u = node;
    down = false;
  }
  for (;;) {
    const int lu = heap_level(u);
    int c, l = 0;
    if (down) {
      if (lu == h) return u;  // a leaf: visit it
      c = 2 * u + (qp[lu % t.d] < __ldg(t.split + u) ? 1 : 2);  // near
    } else {
      // the far child at the deepest level with a clear bit
      const uint32_t open = ~mask & ((1u << lu) - 1u);
      if (open == 0u) return kDone;
      l = 31 - __clz(open);
      const int p = ancestor(u, lu, l + 1);  // path node at level l + 1
      c = 4 * ((p - 1) >> 1) + 3 - p;        // its sibling
      mask |= 1u << l;  // finished from here on: pruned now, or entered now
                        // (then it is on the path)
    }
    const bool pass = B::keep(bx.box(t, c), bound);
    if (down) {
      u = c;  // a pruned near child is finished without a visit; its far
      down = pass;  // sibling (clear bit) is next in line
    } else if (pass) {
      u = c;
      mask &= (2u << l) - 1u;  // levels below l: a new path
      down = true;
    }
  }
}

}  // namespace bkd
