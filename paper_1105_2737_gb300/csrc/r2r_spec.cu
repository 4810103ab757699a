// The Neumann / Dirichlet line kernel compiled for fixed geometries: 512
// threads of 16 points, transform length 2N = 2^LNF = 512 .. 8192 with
// 2^(13 - LNF) line pairs per CTA, for the noise launch (rows) and the strided
// launches (see r2r.cuh).
#include "r2r.cuh"

namespace grf {

namespace {

template <int SRC, int BC, int LNF>
cudaError_t r2r_spec_t(const R2rArgs& a, cudaStream_t s) {
  return r2r::launch_r2r_t<16, SRC, BC, LNF, (1 << (13 - LNF))>(a, s);
}

template <int SRC, int BC>
bool r2r_spec_ln(const R2rArgs& a, cudaStream_t s, cudaError_t* err) {
  switch (a.logNF) {
    case 9: *err = r2r_spec_t<SRC, BC, 9>(a, s); return true;
    case 10: *err = r2r_spec_t<SRC, BC, 10>(a, s); return true;
    case 11: *err = r2r_spec_t<SRC, BC, 11>(a, s); return true;
    case 12: *err = r2r_spec_t<SRC, BC, 12>(a, s); return true;
    case 13: *err = r2r_spec_t<SRC, BC, 13>(a, s); return true;
    default: return false;
  }
}

}  // namespace

bool launch_r2r_spec(int src, const R2rArgs& a, cudaStream_t s, cudaError_t* err) {
  if (a.logNF < 9 || a.logNF > 13 || (2 << (a.logNF - 1)) != 2 * a.N || a.C != (1 << (13 - a.logNF)) ||
      a.logC != 13 - a.logNF)
    return false;
  const bool dir = a.bc == 2;
  if (src == r2r::R2R_NOISE_ROWS)
    return dir ? r2r_spec_ln<r2r::R2R_NOISE_ROWS, 2>(a, s, err) : r2r_spec_ln<r2r::R2R_NOISE_ROWS, 1>(a, s, err);
  if (src == r2r::R2R_LOAD_STRIDED)
    return dir ? r2r_spec_ln<r2r::R2R_LOAD_STRIDED, 2>(a, s, err) : r2r_spec_ln<r2r::R2R_LOAD_STRIDED, 1>(a, s, err);
  return false;
}

}  // namespace grf
