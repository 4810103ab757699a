// The __global__ kernels of the FP32 passes (templates), shared by the
// translation units that instantiate them (fft_kernels.cu, noise_kernels.cu),
// and the launch helper of the column kernels.
#pragma once
#include "bodies.cuh"

namespace grf {

// LN, CC != 0: the transform length 2^LN and the columns (rows) per CTA are
// compile-time constants, so the stage loop unrolls and every shared-memory
// and twiddle address of the exchanges is a constant offset.  These forms are
// compiled for the 256-thread radix-16 geometries (C N = 4096) and chosen by
// the launchers; LN = CC = 0 is the general kernel.
template <int P, int SRC, int MODE, int PAIR, int LN = 0, int CC = 0>
__global__ void __launch_bounds__(kMaxThreads<P>, kMinBlocks<P>) col_kernel(ColArgs a) {
  extern __shared__ float2 sm[];
  if constexpr (PAIR) {
    col_body_pair<P, SRC, MODE, LN, CC>(a, CtaCoordsHW{}, blockDim.x, sm);
  } else {
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    col_body<P, SRC, MODE, LN, CC>(a, blockIdx.x, blockIdx.y, blockIdx.z, blk, blockDim.x, sm);
  }
}

template <int P, int SRC, int MODE, int LN = 0, int CC = 0, int TT = 0, int BZ = -1>
__global__ void __launch_bounds__(kMaxThreads<P>, kMinBlocks<P>) row_kernel(RowArgs a) {
  extern __shared__ float2 sm[];
  row_body<P, SRC, MODE, LN, CC, TT, BZ>(a, blockIdx.x, blockDim.x, sm);
}

// log2 N if (N, C) is one of the compile-time radix-16 geometries (C N = 4096,
// 256 threads, N in [lo, hi]), else 0.
inline int spec_ln(int P, int N, int C, int lo, int hi) {
  if (P != 16 || N < lo || N > hi || (N & (N - 1)) || (int64_t)C * N != 4096) return 0;
  int l = 0;
  while ((1 << l) < N) ++l;
  return l;
}

// Grid-stride forms of the two 2-D/3-D passes: `gridDim.x` CTAs walk all
// tiles, so a small grid leaves room on every SM for another kernel's CTAs
// (the pipelined schedule runs one CTA per SM of each pass side by side).
template <int P, int SRC, int MODE, int PAIR>
__global__ void __launch_bounds__(512) col_kernel_gs(ColArgs a, int gx, int gy, int gz) {
  extern __shared__ float2 sm[];
  const int64_t n = (int64_t)gx * gy * gz;
  for (int64_t t = blockIdx.x; t < n; t += gridDim.x) {
    const int bx = (int)(t % gx);
    const int64_t r = t / gx;
    if constexpr (PAIR) col_body_pair<P, SRC, MODE>(a, CtaCoordsVal{bx, (int)(r % gy), r / gy}, blockDim.x, sm);
    else col_body<P, SRC, MODE>(a, bx, (int)(r % gy), r / gy, t, blockDim.x, sm);
    __syncthreads();
  }
}

template <int P, int SRC, int MODE>
__global__ void __launch_bounds__(512) row_kernel_gs(RowArgs a, int64_t ntiles) {
  extern __shared__ float2 sm[];
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    row_body<P, SRC, MODE>(a, t, blockDim.x, sm);
    __syncthreads();
  }
}

template <int P>
__global__ void __launch_bounds__(256, 3) fourstep_stage1(FourStepArgs a) {
  extern __shared__ float2 sm[];
  fourstep1_body<P>(a, blockIdx.x, blockIdx.z, blockDim.x, sm);
}

// LN, CC != 0: compile-time transform length 2^LN and CC columns per CTA
// (fourstep_spec.cu).
template <int P, int LN = 0, int CC = 0>
__global__ void __launch_bounds__(256, 3) fourstep_stage1_pair(FourStepArgs a) {
  extern __shared__ float2 sm[];
  fourstep1_pair_body<P, LN, CC>(a, blockIdx.x, blockIdx.z, blockDim.x, sm);
}

template <int P, int LN = 0, int CC = 0>
__global__ void __launch_bounds__(256, 2) fourstep_stage2(FourStepArgs a) {
  extern __shared__ float2 sm[];
  fourstep2_body<P, LN, CC>(a, blockIdx.x, blockIdx.z, blockDim.x, sm);
}

template <int P, int SRC, int MODE, int PAIR, int LN = 0, int CC = 0>
static cudaError_t launch_col_t(const ColArgs& a, dim3 grid, cudaStream_t s) {
  const int threads = a.C * a.N / P;
  const size_t smem = PAIR ? col_pair_smem_bytes(a.N, a.C) : col_smem_bytes(a.N, a.C);
  auto k = col_kernel<P, SRC, MODE, PAIR, LN, CC>;
  cudaError_t e = prepare_kernel((const void*)k, threads, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int P, int SRC, int MODE, int LN = 0, int CC = 0, int TT = 0, int BZ = -1>
static cudaError_t launch_row_t(const RowArgs& a, dim3 grid, cudaStream_t s) {
  const int threads = a.C * (a.M / P);
  size_t smem = row_smem_bytes(a.M, a.C);
  if (MODE == ROW_R2C_ADJ) {
    const size_t need = (size_t)threads * 3 * sizeof(double);
    if (need > smem) smem = need;
  }
  auto k = row_kernel<P, SRC, MODE, LN, CC, TT, BZ>;
  cudaError_t e = prepare_kernel((const void*)k, threads, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace grf
