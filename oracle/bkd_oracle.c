/*
 * bkd_oracle.c -- binary64 reference for exact k-nearest-neighbour search.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark load this file.  It shares no code,
 * header, table or constant with the CUDA path and includes nothing from it.
 *
 * What it computes (Gieseke et al., "Bigger Buffer k-d Trees on
 * Multi-Many-Core Systems"):
 *
 *   Sec. 2.2, problem statement: for every query q in Q, the k >= 1 reference
 *   points of P closest to q in Euclidean distance.  Squared distances are
 *   returned.  Every distance is formed in binary64 from the float32 inputs,
 *       D(q, x) = sum_{j=0}^{d-1} ((double)q_j - (double)x_j)^2,
 *   with one rounding per subtraction, per product and per addition, the
 *   terms added in order j = 0, 1, ..., d-1, starting from 0.0.  (The file is
 *   compiled with -ffp-contract=off so that no product is fused into a sum.)
 *   Candidates are ordered by the key (D, original index): the smaller index
 *   wins a tie.  Besides the k nearest, each query also reports the
 *   (k+1)-th distance (+inf when k == n), which the parity tests use to find
 *   queries whose k-th and (k+1)-th neighbours are too close to tell apart.
 *
 *   bkdo_brute  -- the plain definition: every reference point is scored and
 *                  the k+1 smallest keys are kept (cost O(n m (d + k)),
 *                  Sec. 2.2).
 *
 *   bkdo_tree_build / bkdo_tree_query -- the classical k-d tree of Sec. 2.3:
 *                  the node at level i splits its points at the median of
 *                  dimension i mod d into two halves of (almost) equal size;
 *                  splitting stops at height h, so there are 2^h leaves and
 *                  2^h - 1 split values kept pointer-less in heap order (node
 *                  v has children 2v+1 and 2v+2).  A query first walks down to
 *                  the cell that contains it, then on the way back up visits
 *                  the far child of a node when the squared distance to that
 *                  node's splitting hyperplane does not exceed the current
 *                  (k+1)-th best distance, else prunes it (Sec. 2.3).
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *   - "median" for an even count: a node over leaf-structure positions
 *     [lo, hi) puts the floor((hi-lo)/2) smallest points, by the key
 *     (x_s, original index), at positions [lo, mid) with mid = lo +
 *     floor((hi-lo)/2); the split value is x_s of the point at position mid.
 *     Leaf sizes then differ by at most one.
 *   - descent: q_s < split goes left, otherwise right.
 *   - pruning: the far child is visited iff plane^2 <= current (k+1)-th
 *     distance (the paper's "less than", made non-strict so that a point at
 *     exactly the current bound with a smaller index is not skipped).
 *   - the search keeps k+1 candidates so that the (k+1)-th distance is exact.
 *
 * The median selection is a plain quickselect over whole rows (coordinates
 * plus original index), written here from the textbook; any linear-time
 * selection gives the same partition because the key (x_s, index) is unique.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- distance */

static double sqdist64(const float* q, const float* x, int d) {
  double acc = 0.0;
  for (int j = 0; j < d; ++j) {
    double t = (double)q[j] - (double)x[j];
    acc = acc + t * t;
  }
  return acc;
}

/* -------------------------------------------------- bounded candidate list */

typedef struct {
  double dist;
  int64_t idx;
} cand_t;

static int cand_less(double da, int64_t ia, double db, int64_t ib) {
  return da < db || (da == db && ia < ib);
}

/* Keeps the K smallest keys seen so far in L[0..*cnt), ascending. */
static void offer(cand_t* L, int* cnt, int K, double dist, int64_t idx) {
  int pos;
  if (*cnt == K) {
    if (!cand_less(dist, idx, L[K - 1].dist, L[K - 1].idx)) return;
    pos = K - 1;
  } else {
    pos = (*cnt)++;
  }
  while (pos > 0 && cand_less(dist, idx, L[pos - 1].dist, L[pos - 1].idx)) {
    L[pos] = L[pos - 1];
    --pos;
  }
  L[pos].dist = dist;
  L[pos].idx = idx;
}

static void emit(const cand_t* L, int cnt, int k, int64_t* out_idx,
                 double* out_dist, double* out_next) {
  for (int j = 0; j < k; ++j) {
    out_idx[j] = j < cnt ? L[j].idx : -1;
    out_dist[j] = j < cnt ? L[j].dist : INFINITY;
  }
  *out_next = cnt > k ? L[k].dist : INFINITY;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

int bkdo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------- brute force */

/* Returns 0, or -1 on bad arguments / allocation failure. */
int bkdo_brute(const float* P, int64_t n, int d, const float* Q, int64_t m,
               int k, int64_t* out_idx, double* out_dist, double* out_next,
               int nthreads) {
  if (!P || !Q || !out_idx || !out_dist || !out_next) return -1;
  if (n < 1 || d < 1 || m < 0 || k < 1 || k > n) return -1;
  const int K = k + 1;
  int failed = 0;
  set_threads(nthreads);
#pragma omp parallel
  {
    cand_t* L = (cand_t*)malloc(sizeof(cand_t) * (size_t)K);
    if (!L) {
#pragma omp atomic write
      failed = 1;
    }
#pragma omp for schedule(dynamic, 16)
    for (int64_t qi = 0; qi < m; ++qi) {
      if (!L) continue;
      const float* q = Q + qi * d;
      int cnt = 0;
      for (int64_t i = 0; i < n; ++i)
        offer(L, &cnt, K, sqdist64(q, P + i * d, d), i);
      emit(L, cnt, k, out_idx + qi * k, out_dist + qi * k, out_next + qi);
    }
    free(L);
  }
  return failed ? -1 : 0;
}

/* ------------------------------------------------------- k-d tree: build */

/* Rows of the working copy: coordinates pts[pos*d .. pos*d+d) and original
 * index perm[pos].  Ordering key for dimension s: (pts[pos*d+s], perm[pos]). */
typedef struct {
  float* pts;
  int64_t* perm;
  int d;
} rows_t;

static int row_less(const rows_t* r, int64_t a, int64_t b, int s) {
  float xa = r->pts[a * r->d + s], xb = r->pts[b * r->d + s];
  return xa < xb || (xa == xb && r->perm[a] < r->perm[b]);
}

static void row_swap(rows_t* r, int64_t a, int64_t b) {
  if (a == b) return;
  float* pa = r->pts + a * r->d;
  float* pb = r->pts + b * r->d;
  for (int j = 0; j < r->d; ++j) {
    float t = pa[j];
    pa[j] = pb[j];
    pb[j] = t;
  }
  int64_t t = r->perm[a];
  r->perm[a] = r->perm[b];
  r->perm[b] = t;
}

/* Rearranges rows [lo, hi) so that the row at position kpos is the one of
 * rank kpos - lo by the dimension-s key, rows before it rank lower and rows
 * after it rank higher.  Quickselect with a median-of-three pivot. */
static void select_rows(rows_t* r, int64_t lo, int64_t hi, int64_t kpos,
                        int s) {
  while (hi - lo > 1) {
    int64_t a = lo, b = lo + (hi - lo) / 2, c = hi - 1;
    /* median of three positions -> move to hi-1 as the pivot */
    if (row_less(r, b, a, s)) row_swap(r, a, b);
    if (row_less(r, c, a, s)) row_swap(r, a, c);
    if (row_less(r, c, b, s)) row_swap(r, b, c);
    row_swap(r, b, hi - 1); /* pivot = median, now at hi-1 */
    int64_t store = lo;
    for (int64_t i = lo; i < hi - 1; ++i)
      if (row_less(r, i, hi - 1, s)) row_swap(r, i, store++);
    row_swap(r, store, hi - 1); /* pivot in its final place */
    if (store == kpos) return;
    if (kpos < store)
      hi = store;
    else
      lo = store + 1;
  }
}

typedef struct {
  rows_t rows;
  int h;
  float* split;       /* 2^h - 1, heap order */
  int64_t* leaf_lo;   /* 2^h + 1 leaf bounds in the leaf structure */
} build_t;

static void build_node(build_t* B, int64_t lo, int64_t hi, int level,
                       int64_t node) {
  if (level == B->h) {
    int64_t leaf = node - (((int64_t)1 << B->h) - 1);
    B->leaf_lo[leaf] = lo;
    if (leaf == ((int64_t)1 << B->h) - 1) B->leaf_lo[leaf + 1] = hi;
    return;
  }
  int s = level % B->rows.d;
  int64_t mid = lo + (hi - lo) / 2;
  select_rows(&B->rows, lo, hi, mid, s);
  B->split[node] = B->rows.pts[mid * B->rows.d + s];
#pragma omp task if (hi - lo > 65536)
  build_node(B, lo, mid, level + 1, 2 * node + 1);
#pragma omp task if (hi - lo > 65536)
  build_node(B, mid, hi, level + 1, 2 * node + 2);
#pragma omp taskwait
}

/* Builds the tree of height h over P (n x d, row-major).  Outputs:
 *   split[2^h - 1]      split values in heap order
 *   perm[n]             original index of leaf-structure position pos
 *   pts[n*d]            the rearranged points (the leaf structure)
 *   leaf_lo[2^h + 1]    leaf l covers positions [leaf_lo[l], leaf_lo[l+1])
 * Returns 0, or -1 on bad arguments (including 2^h > n). */
int bkdo_tree_build(const float* P, int64_t n, int d, int h, float* split,
                    int64_t* perm, float* pts, int64_t* leaf_lo,
                    int nthreads) {
  if (!P || !split || !perm || !pts || !leaf_lo) return -1;
  if (n < 1 || d < 1 || h < 0 || h > 40) return -1;
  if (((int64_t)1 << h) > n) return -1;
  memcpy(pts, P, sizeof(float) * (size_t)(n * d));
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  build_t B;
  B.rows.pts = pts;
  B.rows.perm = perm;
  B.rows.d = d;
  B.h = h;
  B.split = split;
  B.leaf_lo = leaf_lo;
  set_threads(nthreads);
#pragma omp parallel
#pragma omp single
  build_node(&B, 0, n, 0, 0);
  return 0;
}

/* ------------------------------------------------------ k-d tree: search */

typedef struct {
  int d, h;
  const float* split;
  const int64_t* perm;
  const float* pts;
  const int64_t* leaf_lo;
} tree_t;

static void search_node(const tree_t* T, const float* q, int64_t node,
                        int level, cand_t* L, int* cnt, int K,
                        int64_t* leaves_visited) {
  if (level == T->h) {
    int64_t leaf = node - (((int64_t)1 << T->h) - 1);
    ++*leaves_visited;
    for (int64_t pos = T->leaf_lo[leaf]; pos < T->leaf_lo[leaf + 1]; ++pos)
      offer(L, cnt, K, sqdist64(q, T->pts + pos * T->d, T->d), T->perm[pos]);
    return;
  }
  int s = level % T->d;
  float sv = T->split[node];
  int64_t near_child = q[s] < sv ? 2 * node + 1 : 2 * node + 2;
  int64_t far_child = q[s] < sv ? 2 * node + 2 : 2 * node + 1;
  search_node(T, q, near_child, level + 1, L, cnt, K, leaves_visited);
  double t = (double)q[s] - (double)sv;
  double plane = t * t;
  double bound = *cnt < K ? INFINITY : L[K - 1].dist;
  if (plane <= bound)
    search_node(T, q, far_child, level + 1, L, cnt, K, leaves_visited);
}

/* k nearest neighbours of every query through the tree built above.
 * out_leaves[m] (optional, may be NULL) receives the number of leaves each
 * query visited.  Returns 0 or -1. */
int bkdo_tree_query(int64_t n, int d, int h, const float* split,
                    const int64_t* perm, const float* pts,
                    const int64_t* leaf_lo, const float* Q, int64_t m, int k,
                    int64_t* out_idx, double* out_dist, double* out_next,
                    int64_t* out_leaves, int nthreads) {
  if (!split || !perm || !pts || !leaf_lo || !Q || !out_idx || !out_dist ||
      !out_next)
    return -1;
  if (n < 1 || d < 1 || h < 0 || m < 0 || k < 1 || k > n) return -1;
  tree_t T = {d, h, split, perm, pts, leaf_lo};
  const int K = k + 1;
  int failed = 0;
  set_threads(nthreads);
#pragma omp parallel
  {
    cand_t* L = (cand_t*)malloc(sizeof(cand_t) * (size_t)K);
    if (!L) {
#pragma omp atomic write
      failed = 1;
    }
#pragma omp for schedule(dynamic, 16)
    for (int64_t qi = 0; qi < m; ++qi) {
      if (!L) continue;
      int cnt = 0;
      int64_t visited = 0;
      search_node(&T, Q + qi * d, 0, 0, L, &cnt, K, &visited);
      emit(L, cnt, k, out_idx + qi * k, out_dist + qi * k, out_next + qi);
      if (out_leaves) out_leaves[qi] = visited;
    }
    free(L);
  }
  return failed ? -1 : 0;
}

/* binary64 squared distances of explicit (query, reference) pairs, for
 * checking returned indices: out[i] = D(Q[qi[i]], P[pi[i]]). */
int bkdo_pair_dist(const float* P, int64_t n, int d, const float* Q, int64_t m,
                   const int64_t* qi, const int64_t* pi, int64_t npairs,
                   double* out) {
  if (!P || !Q || !qi || !pi || !out || d < 1) return -1;
  for (int64_t i = 0; i < npairs; ++i) {
    if (qi[i] < 0 || qi[i] >= m || pi[i] < 0 || pi[i] >= n) return -1;
    out[i] = sqdist64(Q + qi[i] * d, P + pi[i] * d, d);
  }
  return 0;
}
