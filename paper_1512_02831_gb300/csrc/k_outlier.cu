// k_outlier.cu -- the proximity-based outlier score of Sec. 4.3: every
// reference point is ranked by its average (Euclidean) distance to its k
// nearest neighbours among the other reference points -- the all-nearest-
// neighbours problem, a query set equal to the reference set.
//
// The queries are the tree's own points, read back from the leaf structure
// (quads + orig) in original order; each is searched with k + 1 neighbours
// (the point itself is normally its own nearest, at distance 0) and the
// score drops the point's own index from its row -- or, when exact
// duplicates with smaller indices fill the row so that the point itself is
// not in it, the last entry -- and averages the square roots of the k
// squared distances that remain.
#include "bkd_internal.h"

namespace bkd {
namespace {

__global__ void inverse_kernel(const int64_t* __restrict__ orig,
                               int64_t slots, int64_t* __restrict__ inv) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= slots) return;
  const int64_t i = orig[s];
  if (i >= 0) inv[i] = s;
}

__global__ void gather_kernel(const float* __restrict__ pts, int Dp, int d,
                              const int64_t* __restrict__ inv, int64_t i0,
                              int64_t m, float* __restrict__ Q) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int64_t s = inv[i0 + r];
  const float* quad = pts + (s >> 2) * 4 * Dp + (s & 3);
  for (int i = 0; i < d; ++i) Q[r * d + i] = quad[4 * i];
}

__global__ void score_kernel(const int64_t* __restrict__ idx,
                             const float* __restrict__ dist, int64_t i0,
                             int64_t m, int k, float* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int K = k + 1;
  const int64_t self = i0 + r;
  int skip = K - 1;  // the last entry, unless the point itself is listed
  for (int j = 0; j < K; ++j)
    if (idx[r * K + j] == self) {
      skip = j;
      break;
    }
  double sum = 0.0;
  for (int j = 0; j < K; ++j)
    if (j != skip) sum += (double)sqrtf(dist[r * K + j]);
  out[r] = (float)(sum / k);
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_inverse(const int64_t* orig, int64_t slots, int64_t* inv,
                           cudaStream_t s) {
  if (slots <= 0) return cudaSuccess;
  inverse_kernel<<<blocks(slots, 256), 256, 0, s>>>(orig, slots, inv);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float* pts, int Dp, int d, const int64_t* inv,
                          int64_t i0, int64_t m, float* Q, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  gather_kernel<<<blocks(m, 256), 256, 0, s>>>(pts, Dp, d, inv, i0, m, Q);
  return cudaGetLastError();
}

cudaError_t launch_score(const int64_t* idx, const float* dist, int64_t i0,
                         int64_t m, int k, float* out, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  score_kernel<<<blocks(m, 256), 256, 0, s>>>(idx, dist, i0, m, k, out);
  return cudaGetLastError();
}

}  // namespace bkd
