// The noise + axis-1 pass compiled for fixed radix-16 geometries: transform
// length N = 256 .. 4096 with 4096 / N columns (or column pairs) per CTA, 256
// threads (see pass_kernels.cuh).  Both the pair form (the 2-D last column
// pass) and the plain form (the 3-D first pass).
#include "pass_kernels.cuh"

namespace grf {

namespace {

template <int PAIR, int LN>
cudaError_t noise_spec_t(const ColArgs& a, dim3 grid, cudaStream_t s) {
  return launch_col_t<16, COL_NOISE, COL_INV, PAIR, LN, (4096 >> LN)>(a, grid, s);
}

template <int PAIR>
bool noise_spec(int ln, const ColArgs& a, dim3 grid, cudaStream_t s, cudaError_t* err) {
  switch (ln) {
    case 8: *err = noise_spec_t<PAIR, 8>(a, grid, s); return true;
    case 9: *err = noise_spec_t<PAIR, 9>(a, grid, s); return true;
    case 10: *err = noise_spec_t<PAIR, 10>(a, grid, s); return true;
    case 11: *err = noise_spec_t<PAIR, 11>(a, grid, s); return true;
    case 12: *err = noise_spec_t<PAIR, 12>(a, grid, s); return true;
    default: return false;
  }
}

}  // namespace

bool launch_col_noise_spec(int P, const ColArgs& a, dim3 grid, cudaStream_t s, cudaError_t* err) {
  if (launch_noise_pair_fast(P, a, grid, s, err)) return true;
  const int ln = spec_ln(P, a.N, a.C, 256, 4096);
  if (!ln) return false;
  return a.zpair ? noise_spec<1>(ln, a, grid, s, err) : noise_spec<0>(ln, a, grid, s, err);
}

}  // namespace grf
