// probe.cu -- test support: the BF16 screen's tensor-core contraction on
// caller-given operands.
//
// The screen's safety bound (k_screen.cu) rests on one hardware property
// that no IEEE rule fixes: how far the fp32 accumulation inside one bf16
// tensor-core MMA may stray from the exact sum of its products.  This entry
// point runs the very instruction the screen issues (mma.sync m16n8k16, bf16
// inputs, fp32 accumulator) on operands chosen by a test, so that the test
// can compare every result with the exact sum and check the accumulation
// model the bound assumes.
#include <cuda_runtime.h>

#include "bkd.h"
#include "bkd_internal.h"

namespace bkd {
namespace {

// One warp per instance: D = C + A B^T with A 16 x 16, Bt 8 x 16 (row c of
// Bt is column c of B), C and D 16 x 8, bf16 bit patterns for A and Bt.
// Fragments follow the m16n8k16 layout: lane (g, t) = (lane / 4, lane % 4)
// holds A rows g and g + 8, k pairs (2t, 2t+1) and (2t+8, 2t+9); B column g,
// the same k pairs; accumulator rows g, g + 8, columns 2t, 2t+1.
__global__ void mma_probe_kernel(int count, const uint16_t* __restrict__ A,
                                 const uint16_t* __restrict__ Bt,
                                 const float* __restrict__ C,
                                 float* __restrict__ D) {
  const int inst = blockIdx.x;
  if (inst >= count) return;
  const int lane = threadIdx.x, g = lane >> 2, t = lane & 3;
  const uint16_t* a = A + (size_t)inst * 256;
  const uint16_t* b = Bt + (size_t)inst * 128;
  const float* c = C + (size_t)inst * 128;
  float* d = D + (size_t)inst * 128;
  auto pair = [](const uint16_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 16);
  };
  const uint32_t a0 = pair(a + g * 16 + 2 * t),
                 a1 = pair(a + (g + 8) * 16 + 2 * t),
                 a2 = pair(a + g * 16 + 2 * t + 8),
                 a3 = pair(a + (g + 8) * 16 + 2 * t + 8);
  const uint32_t b0 = pair(b + g * 16 + 2 * t),
                 b1 = pair(b + g * 16 + 2 * t + 8);
  float acc[4] = {c[g * 8 + 2 * t], c[g * 8 + 2 * t + 1],
                  c[(g + 8) * 8 + 2 * t], c[(g + 8) * 8 + 2 * t + 1]};
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  d[g * 8 + 2 * t] = acc[0];
  d[g * 8 + 2 * t + 1] = acc[1];
  d[(g + 8) * 8 + 2 * t] = acc[2];
  d[(g + 8) * 8 + 2 * t + 1] = acc[3];
}

}  // namespace
}  // namespace bkd

extern "C" int bkd_probe_mma(int kind, int count, const uint16_t* A,
                             const uint16_t* Bt, const float* C, float* D) {
  using namespace bkd;
  set_error(BKD_OK, "");
  if (kind != 0)
    return set_error(BKD_EINVAL, "unknown probe kind %d", kind);
  if (count < 0 || count > (1 << 20))
    return set_error(BKD_EINVAL, "count out of range");
  if (count == 0) return BKD_OK;
  if (!A || !Bt || !C || !D) return set_error(BKD_EINVAL, "NULL argument");
  const size_t na = (size_t)count * 256 * 2, nb = (size_t)count * 128 * 2,
               nc = (size_t)count * 128 * 4;
  char* buf = nullptr;
  cudaError_t e = dev_malloc(&buf, na + nb + 2 * nc);
  if (e != cudaSuccess)
    return set_error(BKD_ENOMEM, "probe buffers: %s", cudaGetErrorString(e));
  uint16_t* dA = reinterpret_cast<uint16_t*>(buf);
  uint16_t* dB = reinterpret_cast<uint16_t*>(buf + na);
  float* dC = reinterpret_cast<float*>(buf + na + nb);
  float* dD = reinterpret_cast<float*>(buf + na + nb + nc);
  int rc = BKD_OK;
  if (cudaMemcpy(dA, A, na, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dB, Bt, nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dC, C, nc, cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = set_error(BKD_ECUDA, "probe upload failed");
  } else {
    mma_probe_kernel<<<count, 32>>>(count, dA, dB, dC, dD);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, nc, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
      rc = set_error(BKD_ECUDA, "probe failed: %s", cudaGetErrorString(e));
  }
  cudaFree(buf);
  return rc;
}
