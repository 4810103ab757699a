// The Monte Carlo covariance estimator of the paper's 1-D study (§4): for
// fields eta_b sampled on the grid x_j (j = 0..N-1, x_0 the origin),
//   Cov(x_j) = (1 / count) sum_b eta_b(0) eta_b(x_j).
// The sums run in FP64 on FP32 samples; a product of two FP32 values is exact
// in FP64.  Two kernels per chunk of fields: per-block partial sums over FB
// fields for 256 lags at a time, then, per lag, the partials added in a fixed
// order onto the running sums, so the result does not depend on scheduling.
#include "kernels.h"

namespace grf {

namespace {

constexpr int kLagsPerBlock = 256;
constexpr int kFieldsPerBlock = 64;

__global__ void __launch_bounds__(kLagsPerBlock) cov_origin_partial(const float* __restrict__ f, int64_t B, int N,
                                                                    double* __restrict__ partial) {
  const int j = blockIdx.x * kLagsPerBlock + threadIdx.x;
  const int64_t b0 = (int64_t)blockIdx.y * kFieldsPerBlock;
  const int64_t b1 = b0 + kFieldsPerBlock < B ? b0 + kFieldsPerBlock : B;
  if (j >= N) return;
  double acc = 0.0;
  for (int64_t b = b0; b < b1; ++b) {
    const float* row = f + b * N;
    acc += (double)__ldg(row) * (double)__ldg(row + j);
  }
  partial[(int64_t)blockIdx.y * N + j] = acc;
}

__global__ void cov_origin_reduce(const double* __restrict__ partial, int nchunks, int N, double* __restrict__ sums) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += partial[(int64_t)c * N + j];
  sums[j] += s;
}

}  // namespace

int64_t cov_origin_partial_count(int64_t B) { return (B + kFieldsPerBlock - 1) / kFieldsPerBlock; }

cudaError_t launch_cov_origin(const float* f, int64_t B, int N, double* partial, double* sums, cudaStream_t s) {
  if (B < 1 || N < 1 || !f || !partial || !sums) return cudaErrorInvalidValue;
  const int64_t nchunks = cov_origin_partial_count(B);
  if (nchunks > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((N + kLagsPerBlock - 1) / kLagsPerBlock), (unsigned)nchunks);
  cov_origin_partial<<<grid, kLagsPerBlock, 0, s>>>(f, B, N, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cov_origin_reduce<<<(N + 255) / 256, 256, 0, s>>>(partial, (int)nchunks, N, sums);
  return cudaGetLastError();
}

}  // namespace grf
