// Launchers of the specialised 2-D noise pair pass (noise_fast.cuh): one
// kernel per transform length 2^LN (256..4096, 4096 / 2^LN column pairs per
// CTA, 256 threads) and workspace tile T in {1, 2, 4, 8, 16}.
#include "noise_fast.cuh"
#include "pass_kernels.cuh"

namespace grf {

namespace {

template <int LN, int TT>
cudaError_t fast_t(const ColArgs& a, dim3 grid, cudaStream_t s) {
  constexpr int CC = 4096 >> LN;
  const size_t smem = noise_fast_smem_bytes(1 << LN, CC);
  auto k = noise_pair_fast<LN, CC, TT>;
  cudaError_t e = prepare_kernel((const void*)k, 256, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, 256, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LN>
bool fast_ln(const ColArgs& a, dim3 grid, cudaStream_t s, cudaError_t* err) {
  switch (a.T) {
    case 1: *err = fast_t<LN, 1>(a, grid, s); return true;
    case 2: *err = fast_t<LN, 2>(a, grid, s); return true;
    case 4: *err = fast_t<LN, 4>(a, grid, s); return true;
    case 8: *err = fast_t<LN, 8>(a, grid, s); return true;
    case 16: *err = fast_t<LN, 16>(a, grid, s); return true;
    default: return false;
  }
}

}  // namespace

bool launch_noise_pair_fast(int P, const ColArgs& a, dim3 grid, cudaStream_t s, cudaError_t* err) {
  // 2-D pair mode only (axis 1 is the transform axis of the whole field), 32-bit
  // offsets within a field
  if (!a.zpair || !a.plane_is_k1 || a.g.d != 2 || a.g.Nmid != 1 || grid.y != 1) return false;
  if ((int64_t)a.N * (a.g.M + 1) >= (int64_t(1) << 31)) return false;
  const int ln = spec_ln(P, a.N, a.C, 256, 4096);
  if (!ln) return false;
  switch (ln) {
    case 8: return fast_ln<8>(a, grid, s, err);
    case 9: return fast_ln<9>(a, grid, s, err);
    case 10: return fast_ln<10>(a, grid, s, err);
    case 11: return fast_ln<11>(a, grid, s, err);
    case 12: return fast_ln<12>(a, grid, s, err);
    default: return false;
  }
}

}  // namespace grf
