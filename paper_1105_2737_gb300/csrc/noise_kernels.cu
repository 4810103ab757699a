// Launchers of the noise + axis-1 pass (Algorithm 2's first pass: Philox
// noise, the Hermitian arrangement and s_K in registers, then the inverse FFT
// along axis 1), in their own translation unit: each radix is compiled once
// with and once without pair mode, so that each kernel holds only the code it
// runs.
#include "pass_kernels.cuh"

namespace grf {

namespace {

template <int PAIR>
cudaError_t launch_noise_p(int P, const ColArgs& a, dim3 grid, cudaStream_t s) {
  switch (P) {
    case 2: return launch_col_t<2, COL_NOISE, COL_INV, PAIR>(a, grid, s);
    case 4: return launch_col_t<4, COL_NOISE, COL_INV, PAIR>(a, grid, s);
    case 8: return launch_col_t<8, COL_NOISE, COL_INV, PAIR>(a, grid, s);
    case 16: return launch_col_t<16, COL_NOISE, COL_INV, PAIR>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int P>
cudaError_t launch_noise_gs_t(const ColArgs& a, dim3 tiles, int ctas, cudaStream_t s) {
  const int threads = a.C * a.N / P;
  const size_t smem = a.zpair ? col_pair_smem_bytes(a.N, a.C) : col_smem_bytes(a.N, a.C);
  auto k = a.zpair ? col_kernel_gs<P, COL_NOISE, COL_INV, 1> : col_kernel_gs<P, COL_NOISE, COL_INV, 0>;
  cudaError_t e = prepare_kernel((const void*)k, threads, smem);
  if (e != cudaSuccess) return e;
  k<<<ctas, threads, smem, s>>>(a, tiles.x, tiles.y, tiles.z);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_col_noise(int P, const ColArgs& a, dim3 grid, cudaStream_t s) {
  cudaError_t e;
  if (launch_col_noise_spec(P, a, grid, s, &e)) return e;
  return a.zpair ? launch_noise_p<1>(P, a, grid, s) : launch_noise_p<0>(P, a, grid, s);
}

cudaError_t launch_col_noise_gs(int P, const ColArgs& a, dim3 tiles, int ctas, cudaStream_t s) {
  switch (P) {
    case 2: return launch_noise_gs_t<2>(a, tiles, ctas, s);
    case 4: return launch_noise_gs_t<4>(a, tiles, ctas, s);
    case 8: return launch_noise_gs_t<8>(a, tiles, ctas, s);
    case 16: return launch_noise_gs_t<16>(a, tiles, ctas, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace grf
