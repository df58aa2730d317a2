/*
 * bkd.h -- C ABI of the GB300 buffer k-d tree (exact k-nearest neighbours).
 *
 * Method: Gieseke, Oancea, Mahabal, Igel, Heskes, "Bigger Buffer k-d Trees on
 * Multi-Many-Core Systems".  Problem statement (Sec. 2.2): given reference
 * points P = {x_1..x_n} and queries Q = {q_1..q_m} in R^d, return for every
 * query its k >= 1 nearest reference points in Euclidean distance.  The
 * search structure is the buffer k-d tree (Sec. 2.4): a pointer-less top tree
 * of median splits plus a leaf structure holding the rearranged points; the
 * query runs LazySearch (Algorithm 1): repeated FindLeafBatch /
 * buffer insertion / ProcessAllBuffers rounds.  When the leaf structure does
 * not fit in device memory it stays in pinned host memory and is streamed in
 * leaf chunks with double-buffered copies (Sec. 3).
 *
 * Conventions shared by every call:
 *   - Points and queries are float32, row-major: point i occupies
 *     P[i*d .. i*d + d).  Pointers may be host or device memory (detected with
 *     cudaPointerGetAttributes); the caller owns them.
 *   - Results: out_idx (int64) holds 0-based row indices of P; out_dist
 *     (float32) holds SQUARED Euclidean distances.  Both are m x k,
 *     row-major, host or device memory owned by the caller.  Row j lists the
 *     neighbours of query j in ascending order of (exact distance, index): a
 *     tie goes to the smaller index.  The returned float32 distances are
 *     non-decreasing along a row.
 *   - Exactness: indices equal those of a binary64 computation of the same
 *     definition, except where a query's k-th and (k+1)-th neighbours are at
 *     distances too close to separate in binary64 (then any valid k-nearest
 *     set is returned).  Distances agree with binary64 to within
 *     (d + 3) * 2^-24 relative.
 *   - Inputs must be finite with magnitude below 2^60; anything else is
 *     rejected with BKD_EINVAL.
 *   - Every call returns BKD_OK (0) or a negative status; bkd_last_error()
 *     then describes the failure.  On failure the outputs are unspecified and
 *     the tree stays usable unless the status is BKD_ECUDA.
 *   - A tree handle is not thread-safe: one thread (or external locking) per
 *     handle.  Different handles may be used from different threads.
 *   - Work runs on the tree's stream (BKD_OPT_STREAM; by default a stream the
 *     library creates).  Calls return after their results are complete in
 *     the caller's output buffers.
 */
#ifndef BKD_H
#define BKD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define BKD_OK 0
#define BKD_EINVAL (-1)       /* bad argument (null, range, non-finite input) */
#define BKD_ENOMEM (-2)       /* device or pinned host allocation failed      */
#define BKD_ECUDA (-3)        /* CUDA runtime error; the handle should be freed */
#define BKD_ETIMEOUT (-4)     /* a bounded device-side wait ran out           */
#define BKD_EUNSUPPORTED (-5) /* valid request outside the library's limits   */

/* ------------------------------------------------------------------ limits */
#define BKD_MAX_DIM 32        /* d <= BKD_MAX_DIM                              */
#define BKD_MAX_K 63          /* k <= BKD_MAX_K                                */
#define BKD_MAX_HEIGHT 24     /* height <= BKD_MAX_HEIGHT                      */
#define BKD_STATIC_MAX_QUERIES 4096      /* m limit of bkd_query_static      */
#define BKD_STATIC_MAX_HEIGHT 16         /* tree height limit of it          */
#define BKD_STATIC_SCRATCH_BYTES 8388608 /* its static device scratch area   */

/* ----------------------------------------------------------------- options
 * Set with bkd_set_option (after build) or passed as (key, value) pairs to
 * bkd_build_with (at build).  Unknown keys are rejected with BKD_EINVAL. */
enum bkd_option {
  /* cudaStream_t (as an integer) on which all work of the handle runs;
   * 0 selects the library's own stream, a non-blocking stream that is not
   * ordered with the legacy default stream: inputs written there must be
   * complete before the call (synchronise it first, or pass CUDA's handle of
   * that stream, cudaStreamLegacy).  Any time. */
  BKD_OPT_STREAM = 1,
  /* Bytes of device memory the leaf structure may occupy.  If the leaf
   * structure is larger, the tree is built in chunked ("bigger") mode: it
   * stays in pinned host memory and is streamed (Sec. 3.2).  Build only;
   * default: 60% of the device memory free at build time. */
  BKD_OPT_DEVICE_MEM_CAP = 2,
  /* Number N of leaf chunks in chunked mode (Sec. 3.2, "1 < N << n").  0
   * (default) picks the smallest N whose two chunk buffers fit the cap.  A
   * value >= 1 at build forces chunked mode with that N.  Build only. */
  BKD_OPT_CHUNKS = 3,
  /* Maximum number of queries in flight in one LazySearch (the bounded query
   * memory of Sec. 3.2, "Multi-Many-Core Querying"); larger query sets are
   * processed in consecutive slices.  0 (default) = all m at once. */
  BKD_OPT_MAX_ACTIVE = 4,
  /* When at most this many queries remain active, they finish in one launch
   * (one warp per query walks its remaining leaves) instead of one
   * LazySearch round per leaf.  -1 (default) = automatic (8192, growing to
   * 32768 for query sets of 2^24); 0 = never.
   * Results do not depend on it.  Any time. */
  BKD_OPT_TAIL_QUERIES = 5,
  /* Leaf scoring: 0 (default) = float32 for every (query, point) pair;
   * 1 = a BF16 tensor-core screen rejects points that provably cannot enter
   * a candidate list, the rest are scored in float32 -- results identical to
   * 0.  1 at build also prepares the screen data; afterwards 0 / 1 may be
   * switched any time.  Chunked trees: leaf chunks and the warp screen
   * kernel only (the screen operands are streamed with each chunk's
   * points); with BKD_OPT_POINT_CHUNKS=1 or BKD_OPT_SCREEN_KERNEL=1 the
   * build fails with BKD_EUNSUPPORTED. */
  BKD_OPT_PRECISION = 6,
  /* Chunk bounds in chunked mode: 0 (default) = whole leaves (chunk c holds
   * leaves [ceil(c L / N), ceil((c+1) L / N)), L = 2^h), scheduled so that
   * the two chunks resident on the device keep running while they hold
   * buffered queries; 1 = the point chunks of Sec. 3.2, positions
   * [ceil(j n / N), ceil((j+1) n / N)) of the leaf structure (a bound inside
   * a leaf moved down to a multiple of 4 points from the leaf's start), so
   * a leaf may straddle two chunks and its queries are scanned in both;
   * every chunk holding buffered queries is streamed every round.  Results
   * do not depend on it.  Build only (with BKD_OPT_CHUNKS >= 1 or the
   * memory cap). */
  BKD_OPT_POINT_CHUNKS = 7,
  /* Launch shapes (results do not depend on them; any time):
   * queries per work item of a screened round: the warp screen kernel
   * 8..32 in steps of 8 (default 32), the tcgen05 screen kernel 16..128 in
   * steps of 16 (default 128); reset to the default when the kernel is
   * switched */
  BKD_OPT_SCREEN_TILE = 8,
  /* LazySearch rounds queued on a resident tree before the host looks at
   * the counters again, 1..64; 0 (default) = automatic (64 far from the
   * tail threshold, then 16, then 4) */
  BKD_OPT_ROUND_BATCH = 9,
  /* CTAs per SM of the screen kernel, 1..3; 0 (default) = as many as
   * registers, shared and tensor memory allow */
  BKD_OPT_SCREEN_CTAS = 10,
  /* Which BF16 screen kernel runs the screened rounds (both keep the
   * float32 result, Sec. 2.2 exactness; results do not depend on it):
   * 0 (default) = one warp per work item of <= 32 queries, mma.sync
   * m16n8k16 with the accumulators in registers; 1 = tcgen05.mma into
   * tensor memory, 128-point tiles by bulk copy, work items of <= 128
   * queries, survivors rescored by a separate kernel.  At build (with
   * BKD_OPT_PRECISION=1) it picks the point layouts prepared: 0 or 1 that
   * kernel's, 2 both (kernel 0 runs first); afterwards 0 / 1 may be
   * switched any time among the layouts the tree holds (else BKD_EINVAL). */
  BKD_OPT_SCREEN_KERNEL = 11,
  /* Servers on this tree: a batch still running this many LazySearch rounds
   * after its admission has its remaining queries finished by the tail
   * kernel (bounds a batch's latency; results do not depend on it); 0 =
   * never; default 384.  Any time. */
  BKD_OPT_RESCUE_ROUNDS = 12,
  /* Servers on this tree: the buffer trigger of Algorithm 1 -- a round
   * processes a leaf's buffer only when it holds at least this many queries
   * or was deferred 4 rounds in a row; the other buffered queries wait at
   * their leaf (fewer, fuller leaf scans on trees with many leaves; results
   * do not depend on it); 0 (default) = every buffer every round, 0..4096.
   * Any time. */
  BKD_OPT_DEFER_QUERIES = 13
};

/* ------------------------------------------------------------------- stats
 * Counters of the most recent bkd_query on the handle (bkd_get_stat). */
enum bkd_stat {
  BKD_STAT_ROUNDS = 1,         /* LazySearch iterations (Algorithm 1 loop)   */
  BKD_STAT_LEAF_VISITS = 2,    /* (query, leaf) pairs of the LazySearch rounds */
  BKD_STAT_PAIRS = 3,          /* distances scored by the leaf kernel        */
  BKD_STAT_RESORTED = 4,       /* queries re-ordered by binary64 distances   */
  BKD_STAT_FALLBACK = 5,       /* queries re-searched in binary64            */
  BKD_STAT_LEAF_KERNEL_MS = 6, /* summed device time of the leaf kernel      */
  BKD_STAT_CHUNK_BYTES = 7,    /* host-to-device leaf-chunk bytes (chunked)  */
  BKD_STAT_COPY_MS = 8,        /* summed device time of the chunk copies     */
  BKD_STAT_LEAF_LAUNCHES = 9,  /* launches of the leaf kernel                */
  BKD_STAT_KERNEL_LAUNCHES = 10, /* all kernel launches of the query         */
  BKD_STAT_TAIL_QUERIES = 11,  /* queries finished by the tail kernel        */
  BKD_STAT_TAIL_VISITS = 12,   /* (query, leaf) visits of the tail kernel    */
  BKD_STAT_TAIL_PAIRS = 13,    /* distances scored by the tail kernel        */
  BKD_STAT_TAIL_MS = 14,       /* device time of the tail kernel             */
  BKD_STAT_SCREEN_KEPT = 15,   /* pairs the BF16 screen passed to float32    */
  BKD_STAT_SCREEN_PAIRS = 16,  /* pairs the BF16 screen kernel examined      */
  BKD_STAT_SCREEN_MS = 17,     /* device time of the BF16 screen kernel      */
  BKD_STAT_SCREEN_ITEMS = 18,  /* work items (one leaf, <= 128 queries)     */
  BKD_STAT_SCREEN_VISITS = 19, /* (query, leaf) pairs of the screened rounds */
  BKD_STAT_FIND_MS = 20,       /* device time of FindLeafBatch (all rounds)  */
  BKD_STAT_BUCKET_MS = 21,     /* device time of the bucketing (all rounds)  */
  BKD_STAT_EXACT_MS = 22,      /* device time of the binary64 re-check and
                                  fallback search                           */
  BKD_STAT_CHUNK_VISITS = 23,  /* chunked mode: (query, leaf) pairs scanned
                                  (queries waiting in a chunk not brought in
                                  that round are not counted)               */
  BKD_STAT_SCREEN_BYTES = 24,  /* bytes of bf16 operand tiles the screen
                                  streamed from HBM into shared memory      */
  BKD_STAT_SCREEN_QUEUED = 25, /* pairs the screen queued for rescoring     */
  BKD_STAT_SCREEN_OVERFLOW = 26, /* screen items rescored against the whole
                                  leaf (their rescoring queue overflowed)  */
  BKD_STAT_LEAF_BYTES = 27,     /* bytes of the leaf structure the float32
                                  leaf kernel staged in shared memory (one
                                  pass over the leaf per work item)        */
  BKD_STAT_HOST_SYNCS = 28,     /* times the host waited for the device's
                                  round counters (resident trees queue up
                                  to BKD_OPT_ROUND_BATCH rounds per look)  */
  BKD_STAT_FALLBACK_POINTS = 29, /* points the binary64 fallback scanned   */
  BKD_STAT_MAPPED_BYTES = 30    /* chunked trees: point bytes the tail,
                                  re-check and fallback kernels read from
                                  the mapped pinned host leaf structure
                                  (zero-copy, not in chunk_bytes)          */
};

typedef struct bkd_tree bkd_tree; /* opaque; owned by the library */

/* bkd_build -- construction phase (Sec. 2.3 median splits; Sec. 3.1 "build
 * the top tree on the host and store it on the device").
 *   P       n x d float32 reference points, host or device.  Read only during
 *           the call; the library keeps its own rearranged copy.
 *   n       number of points, 1 <= n; 2^height <= n.
 *   d       dimension, 1 <= d <= BKD_MAX_DIM.
 *   height  h: the top tree has 2^h - 1 split values and 2^h leaves, leaf
 *           sizes differ by at most one.  0 <= h <= BKD_MAX_HEIGHT.
 *   out     receives the new handle (NULL on failure).
 * Node v at level i splits its points at the median of dimension i mod d:
 * the floor(size/2) points smallest by (x_{i mod d}, index) go left; the
 * split value is the smallest coordinate of the right half.
 * Errors: BKD_EINVAL, BKD_ENOMEM, BKD_ECUDA, BKD_EUNSUPPORTED. */
int bkd_build(const float* P, int64_t n, int d, int height, bkd_tree** out);

/* bkd_build_with -- bkd_build with build-time options: `options` holds
 * `n_options` (key, value) pairs, keys from enum bkd_option. */
int bkd_build_with(const float* P, int64_t n, int d, int height,
                   const int64_t* options, int n_options, bkd_tree** out);

/* bkd_query -- query phase: LazySearch (Algorithm 1) with FindLeafBatch,
 * buffer insertion and ProcessAllBuffers on the device; in chunked mode
 * ProcessAllBuffers streams the leaf chunks (Sec. 3.2, Brute / Copy / Wait).
 *   t         handle from bkd_build.
 *   Q         m x d float32 queries (same d as the tree), host or device.
 *   m         number of queries, m >= 0 (m == 0 returns at once).
 *   k         neighbours per query, 1 <= k <= min(n, BKD_MAX_K).
 *   out_idx   m x k int64, host or device (caller-owned).
 *   out_dist  m x k float32 squared distances, host or device.
 * Errors: BKD_EINVAL, BKD_ENOMEM, BKD_ECUDA, BKD_ETIMEOUT,
 * BKD_EUNSUPPORTED. */
int bkd_query(bkd_tree* t, const float* Q, int64_t m, int k, int64_t* out_idx,
              float* out_dist);

/* bkd_query_static -- bkd_query that performs no memory allocation.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot call cudaMalloc / cudaFree while answering queries: a process whose
 * device memory is owned entirely by its own pool allocator, or a
 * latency-critical loop that cannot let cudaFree synchronise the device.
 * It runs the same kernels as bkd_query, with its workspace in a fixed
 * BKD_STATIC_SCRATCH_BYTES area of static device memory inside the library
 * (held by every GPU that loads the library until the process exits).
 *   t         handle from bkd_build; must be resident (not chunked) and of
 *             height <= BKD_STATIC_MAX_HEIGHT.
 *   Q         m x d float32 queries in DEVICE memory.
 *   m         0 <= m <= BKD_STATIC_MAX_QUERIES; larger m is rejected with
 *             BKD_EINVAL (split the call or use bkd_query).
 *   k         1 <= k <= min(n, BKD_MAX_K).
 *   out_idx, out_dist  m x k, DEVICE memory, same meaning as bkd_query.
 * Results equal bkd_query's.  Host pointers are rejected (BKD_EINVAL); a
 * chunked tree gives BKD_EUNSUPPORTED.
 * The first call on a device looks up the scratch area's device address
 * (cudaGetSymbolAddress, with the tree's device current); make that first
 * call before any stream capture.  All calls on a device share the one
 * scratch area and each call overwrites it: calls whose GPU work overlaps --
 * from several threads, or on several streams -- race and corrupt each
 * other's results; serialise them. */
int bkd_query_static(bkd_tree* t, const float* Q, int64_t m, int k,
                     int64_t* out_idx, float* out_dist);

/* bkd_outlier_scores -- the proximity-based outlier score of Sec. 4.3 (each
 * point is ranked by the mean distance to its k nearest neighbours: the
 * all-nearest-neighbours problem, queries = the reference points): for
 * every reference point i (original row order),
 *   out_score[i] = (1/k) sum of the Euclidean (not squared) distances from
 *                  x_i to its k nearest neighbours among the OTHER points,
 * neighbours taken under the same (distance, index) order as bkd_query: x_i
 * is searched with k + 1 neighbours and its own index is dropped from the
 * row (if exact duplicates with smaller indices fill the row, x_i is not in
 * it and the last entry is dropped).  Distances are float32 square roots of
 * bkd_query's squared distances, summed in binary64.
 *   t          handle from bkd_build (resident or chunked).
 *   k          1 <= k <= n - 1 and k + 1 <= BKD_MAX_K.
 *   out_score  n float32, host or device memory (caller-owned).
 * Queries run in slices of BKD_OPT_MAX_ACTIVE points (default 2^24).
 * Errors: BKD_EINVAL, BKD_ENOMEM, BKD_ECUDA, BKD_ETIMEOUT,
 * BKD_EUNSUPPORTED. */
int bkd_outlier_scores(bkd_tree* t, int k, float* out_score);

/* ------------------------------------------------------------ test support
 * None of these calls has a counterpart in the paper; they let tests reach
 * failure paths and hardware properties that the query calls depend on. */

/* bkd_test_fail_alloc -- makes the nth device or pinned host allocation made
 * by the library from now on (any handle, any thread) fail as if the memory
 * were exhausted; 0 switches the hook off.  The call that meets the failure
 * returns BKD_ENOMEM and leaves its handle usable (bkd_build frees what it
 * had built).  Errors: BKD_EINVAL (nth < 0). */
int bkd_test_fail_alloc(int64_t nth);

/* bkd_test_host_screen -- the host half of bkd_build(P, n, d, height) with
 * BKD_OPT_PRECISION=1, without a GPU: the median-split tree (Sec. 2.3), the
 * bounding box of every heap node, and the BF16 warp screen's operands and
 * per-leaf bounds, computed by the functions bkd_build uses and written to
 * caller buffers (all host memory, caller-owned).
 *   P, n, d, height  as bkd_build (P host memory).
 *   shape    out: int64[8] = {lcap, stride, kh, words, Dp, tiles, tc_kh,
 *            tc_elems}: slots per leaf (largest leaf rounded up to 4),
 *            screen rows per leaf (lcap rounded up to 32), k-halves of 16
 *            bf16 slots, uint32 words of the operand array, padded
 *            dimension; then for the tcgen05 kernel's operands: 128-row
 *            tiles per leaf, k-halves, bf16 elements of tc_words.
 *   split    float[max(2^h - 1, 1)]: split values in heap order.
 *   leaf_lo  int64[2^h + 1]: leaf l holds tree positions [leaf_lo[l],
 *            leaf_lo[l+1]).
 *   perm     int64[n]: the row of P at each tree position.
 *   box      float[(2^(h+1) - 1) * 2 Dp]: per heap node its minimum row and
 *            then its maximum row (dimensions d..Dp-1 are [0, 0]).
 *   words    uint32[words]: per leaf and k-half, stride rows of 8 words in
 *            the screen's fragment order; a word holds two bf16 slots (low
 *            half first); slots 0..d-1 of a row are the point's offset from
 *            the leaf centre, slots d and d+1 the split of its squared norm,
 *            the rest 0; rows past the leaf's points have slot d = +inf.
 *   center   float[2^h * d]: per leaf the midpoint of its bounding box.
 *   bmax     float[2^h]: per leaf an upper bound of the Euclidean norm
 *            ||w - w_hat|| over its points (w = x - centre, exact; w_hat
 *            its bf16 operand).
 *   pnmax    float[2^h]: per leaf an upper bound of ||w_hat||^2.
 *   tc_words uint16[tc_elems]: the tcgen05 kernel's operand tiles, per leaf
 *            `tiles` tiles of 128 rows x 16 tc_kh bf16, row r's slots
 *            8 g .. 8 g + 7 at byte (r / 8) 256 tc_kh + 128 g + 16 (r % 8)
 *            of its tile; a row holds the same offsets and norm split as
 *            above, then 1.0 in slots d+2 .. d+4; padding rows slot d =
 *            +inf.  Its centre and bounds equal the ones above (checked:
 *            BKD_EINVAL otherwise).
 * Pass all of split ... tc_words to fill them, or none of them to learn
 * shape only.  Errors: BKD_EINVAL, BKD_ENOMEM. */
int bkd_test_host_screen(const float* P, int64_t n, int d, int height,
                         int64_t* shape, float* split, int64_t* leaf_lo,
                         int64_t* perm, float* box, uint32_t* words,
                         float* center, float* bmax, float* pnmax,
                         uint16_t* tc_words);

/* bkd_probe_mma -- runs the warp screen kernel's tensor-core instruction
 * (kind 0: mma.sync m16n8k16, bf16 inputs, fp32 accumulation) on `count`
 * instances:
 * D = C + A Bt^T, with A count x 16 x 16 and Bt count x 8 x 16 bf16 bit
 * patterns (row-major; row c of Bt is column c of the B operand), C and D
 * count x 16 x 8 float32, all HOST memory.  The screen's error bound
 * (Sec. 2.2 exactness of the answer) assumes how far this accumulation may
 * stray from the exact sum; tests compare D with exact sums.
 * Errors: BKD_EINVAL, BKD_ENOMEM, BKD_ECUDA. */
int bkd_probe_mma(int kind, int count, const uint16_t* A, const uint16_t* Bt,
                  const float* C, float* D);

/* bkd_probe_umma -- the BF16 screen's Blackwell tensor-core path (operands
 * staged in shared memory in the screen's layout, kh chained tcgen05.mma of
 * kind::f16 with K = 16, M = 128, N = n, fp32 accumulator in tensor memory,
 * read back with tcgen05.ld) on `count` instances: D = A Bt^T with A
 * count x 128 x 16 kh and Bt count x n x 16 kh bf16 bit patterns
 * (row-major), D count x 128 x n float32, all HOST memory; 16 <= n <= 256,
 * n a multiple of 16, 1 <= kh <= 3.  Tests compare D with exact sums to pin
 * the accumulation model of the screen's error bound.
 * Errors: BKD_EINVAL, BKD_ENOMEM, BKD_ECUDA, BKD_ETIMEOUT. */
int bkd_probe_umma(int n, int kh, int count, const uint16_t* A,
                   const uint16_t* Bt, float* D);

/* bkd_set_option -- sets a run-time option (enum bkd_option) on a handle.
 * Build-only keys are rejected with BKD_EINVAL. */
int bkd_set_option(bkd_tree* t, int key, int64_t value);

/* bkd_get_stat -- reads a counter of the last query (enum bkd_stat). */
int bkd_get_stat(const bkd_tree* t, int key, double* value);

/* bkd_tree_shape -- n, d, height, chunked mode (0/1) and chunk count N of a
 * handle.  Any output pointer may be NULL. */
int bkd_tree_shape(const bkd_tree* t, int64_t* n, int* d, int* height,
                   int* chunked, int* chunks);

/* bkd_export_tree -- copies the tree to caller-owned HOST arrays (for
 * inspection and tests):
 *   split    2^h - 1 float32 split values in heap order (node v has children
 *            2v+1 and 2v+2); may be NULL
 *   leaf_lo  2^h + 1 int64: leaf l holds leaf-structure positions
 *            [leaf_lo[l], leaf_lo[l+1]); may be NULL
 *   perm     n int64: original index of leaf-structure position p; may be
 *            NULL */
int bkd_export_tree(const bkd_tree* t, float* split, int64_t* leaf_lo,
                    int64_t* perm);

/* bkd_free -- releases the handle and all its device / pinned memory.
 * NULL is ignored. */
void bkd_free(bkd_tree* t);

/* bkd_last_error -- message of the last failed call on this thread ("" if
 * none).  The string stays valid until the thread's next bkd_* call. */
const char* bkd_last_error(void);

/* ------------------------------------------------------------------ serving
 * Continuous batching over a resident tree.  The paper's on-the-fly querying
 * (Sec. 3.2: new queries are fetched from the input queue while others are
 * still in flight) made into a request loop: batches of any size and k are
 * queued, admitted into free query slots as earlier batches finish, and every
 * admitted query advances in the SAME LazySearch rounds (FindLeafBatch,
 * buffer insertion, ProcessAllBuffers) -- work of different batches shares
 * every launch.  A batch's results equal a bkd_query of it alone. */
typedef struct bkd_server bkd_server; /* opaque; owned by the library */

enum bkd_batch_status {
  BKD_BATCH_QUEUED = 0,   /* waiting for free query slots                    */
  BKD_BATCH_RUNNING = 1,  /* admitted; its queries are in the rounds         */
  BKD_BATCH_DONE = 2      /* results written to its output buffers           */
  /* a negative status is the error code the batch failed with */
};

/* bkd_serve_open -- a server on tree t (resident, not chunked).
 *   k_max        largest k a batch may ask for, 1 <= k_max <= min(n,
 *                BKD_MAX_K).  Batches are routed by k to list classes of
 *                at most 12, 32 or 64 entries (those up to k_max + 1): a
 *                query carries its class's list, and a class's rounds run
 *                with that list length.
 *   max_queries  query slots of each class: the most queries in flight at
 *                once in a class (device memory per class ~ max_queries x
 *                (4 Dp + 8 kc + 60) bytes, kc the class's largest k).
 *   out          receives the server (NULL on failure).
 * The server uses the tree's stream; do not run bkd_query on the same tree
 * while the server has batches in flight.
 * Errors: BKD_EINVAL, BKD_ENOMEM, BKD_ECUDA, BKD_EUNSUPPORTED. */
int bkd_serve_open(bkd_tree* t, int k_max, int64_t max_queries,
                   bkd_server** out);

/* bkd_serve_submit -- queues a batch (no GPU work).
 *   Q         m x d float32 queries, host or device; must stay valid and
 *             unchanged until the batch is DONE (or failed).
 *   m         0 <= m <= max_queries (m == 0 is DONE at once).
 *   k         1 <= k <= k_max.
 *   out_idx, out_dist  m x k int64 / float32, host or device, written when
 *             the batch completes (same meaning as bkd_query).
 *   ticket    receives the batch's ticket (>= 1).
 * Errors: BKD_EINVAL. */
int bkd_serve_submit(bkd_server* s, const float* Q, int64_t m, int k,
                     int64_t* out_idx, float* out_dist, int64_t* ticket);

/* bkd_serve_step -- admits queued batches (first come, first served) while
 * contiguous free slots fit them, runs ONE LazySearch round over every
 * admitted query, and completes the batches whose queries all finished
 * (binary64 re-check, fallback, results to the caller's buffers).
 *   pending  receives the number of batches not yet completed (queued or
 *            running); may be NULL.
 * A batch whose queries hold a non-finite value fails with BKD_EINVAL
 * (its status) without affecting the others.
 * Errors: BKD_EINVAL (NULL server), BKD_ECUDA, BKD_ETIMEOUT. */
int bkd_serve_step(bkd_server* s, int64_t* pending);

/* bkd_serve_status -- status of a ticket (enum bkd_batch_status, or the
 * negative error code the batch failed with).  A terminal status (DONE or
 * failed) is reported once; afterwards the ticket is unknown (BKD_EINVAL). */
int bkd_serve_status(bkd_server* s, int64_t ticket, int* status);

/* bkd_serve_close -- waits for the device, releases the server (queued and
 * running batches are dropped without results).  Close servers before
 * freeing their tree.  NULL is ignored. */
void bkd_serve_close(bkd_server* s);

#ifdef __cplusplus
}
#endif

#endif /* BKD_H */
