// Measured lane-operation rates of this GPU: the denominators of the ALU view
// of the noise pass's roofline (no counterpart in the paper).  Each kernel runs
// eight independent dependency chains per thread over a grid of 8 CTAs of 256
// threads per SM, long enough (tens of ms) that launch overhead is noise; the
// chains' results are stored so that nothing is optimised away.
//   kind 0: FP32 fused multiply-add (one lane-operation each): the issue rate
//           of the FMA pipes, the ceiling of any instruction mix;
//   kind 1: rounds of Philox4x32 (two 32 x 32 -> 64-bit multiplies and two
//           three-input XORs per chain: four lane-operations; the two key
//           additions of a round are shared by the eight chains);
//   kind 2: the special-function pair of Box-Muller (log2 and reciprocal
//           square root, one lane-operation each).
#include <cuda_runtime.h>
#include <stdint.h>
#include "grf.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_rate(float* sink, float b, float c, int iters) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == 12345.678f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) philox_rate(uint32_t* sink, uint32_t k0in, uint32_t k1in, int iters) {
  uint32_t c0[kChains], c1[kChains], c2[kChains], c3[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    c0[i] = threadIdx.x + i;
    c1[i] = blockIdx.x;
    c2[i] = i;
    c3[i] = 0u;
  }
  uint32_t k0 = k0in, k1 = k1in;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        const uint32_t lo0 = 0xD2511F53u * c0[i], hi0 = __umulhi(0xD2511F53u, c0[i]);
        const uint32_t lo1 = 0xCD9E8D57u * c2[i], hi1 = __umulhi(0xCD9E8D57u, c2[i]);
        c0[i] = hi1 ^ c1[i] ^ k0;
        c1[i] = lo1;
        c2[i] = hi0 ^ c3[i] ^ k1;
        c3[i] = lo0;
      }
    }
  }
  uint32_t s = 0u;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s ^= c0[i] ^ c1[i] ^ c2[i] ^ c3[i];
  if (s == 0x12345678u) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) mufu_rate(float* sink, float b, int iters) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1.5f + 0.01f * (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = rsqrtf(__log2f(a[i]) + b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == 12345.678f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" grf_status grf_alu_peak(int kind, double* ops_per_s, void* stream) {
  if (!ops_per_s || kind < 0 || kind > 2) return GRF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return GRF_ERR_CUDA;
  const int blocks = sms * 8;
  // 8 x 16 x iters steps per thread: at 152 SMs about 2.5e9 FMAs, 4.8e8 Philox
  // rounds or 1.6e8 log / rsqrt pairs, each some tens of ms
  const int iters = kind == 0 ? 64 : (kind == 1 ? 12 : 4);
  void* sink = nullptr;
  if (cudaMalloc(&sink, (size_t)blocks * kThreads * 4) != cudaSuccess) return GRF_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  grf_status st = GRF_OK;
  float ms = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = GRF_ERR_CUDA;
  } else {
    for (int rep = 0; rep < 2 && st == GRF_OK; ++rep) {  // the first launch warms up
      if (rep == 1) cudaEventRecord(e0, s);
      if (kind == 0) fma_rate<<<blocks, kThreads, 0, s>>>((float*)sink, 0.999f, 0.001f, iters);
      else if (kind == 1) philox_rate<<<blocks, kThreads, 0, s>>>((uint32_t*)sink, 7u, 11u, iters);
      else mufu_rate<<<blocks, kThreads, 0, s>>>((float*)sink, 0.25f, iters);
      if (cudaGetLastError() != cudaSuccess) st = GRF_ERR_CUDA;
      if (rep == 1) cudaEventRecord(e1, s);
    }
    if (st == GRF_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = GRF_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (st != GRF_OK || ms <= 0.f) return st != GRF_OK ? st : GRF_ERR_CUDA;
  const double per_step = kind == 0 ? 1.0 : (kind == 1 ? 4.0 + 2.0 / kChains : 2.0);
  const double ops = (double)blocks * kThreads * kChains * 16.0 * (double)iters * per_step;
  *ops_per_s = ops / (ms * 1e-3);
  return GRF_OK;
}
