// The axis-2 pair pass (3-D) and the c2r pass compiled for fixed radix-16
// geometries: length 2^LN with 4096 / 2^LN columns or rows per CTA, 256
// threads (see pass_kernels.cuh); the c2r pass also per workspace tile T.
#include "pass_kernels.cuh"

namespace grf {

namespace {

template <int LN>
cudaError_t load_pair_t(const ColArgs& a, dim3 grid, cudaStream_t s) {
  return launch_col_t<16, COL_LOAD, COL_INV, 1, LN, (4096 >> LN)>(a, grid, s);
}
// the workspace tile T as a compile-time constant (T in {1, 2, 4, 8, 16}) for
// a plan's fields; a batch plan's launch (outputs by field) keeps T at run time
template <int LN>
cudaError_t row_c2r_t(const RowArgs& a, dim3 grid, cudaStream_t s) {
  constexpr int CC = 4096 >> LN;
  if (a.zout) return launch_row_t<16, ROW_LOAD_Z, ROW_C2R, LN, CC, 0, 1>(a, grid, s);
  switch (a.T) {
    case 1: return launch_row_t<16, ROW_LOAD_Z, ROW_C2R, LN, CC, 1, 0>(a, grid, s);
    case 2: return launch_row_t<16, ROW_LOAD_Z, ROW_C2R, LN, CC, 2, 0>(a, grid, s);
    case 4: return launch_row_t<16, ROW_LOAD_Z, ROW_C2R, LN, CC, 4, 0>(a, grid, s);
    case 8: return launch_row_t<16, ROW_LOAD_Z, ROW_C2R, LN, CC, 8, 0>(a, grid, s);
    case 16: return launch_row_t<16, ROW_LOAD_Z, ROW_C2R, LN, CC, 16, 0>(a, grid, s);
    default: return launch_row_t<16, ROW_LOAD_Z, ROW_C2R, LN, CC, 0, 0>(a, grid, s);
  }
}

}  // namespace

bool launch_col_load_pair_spec(int P, const ColArgs& a, dim3 grid, cudaStream_t s, cudaError_t* err) {
  switch (spec_ln(P, a.N, a.C, 256, 4096)) {
    case 8: *err = load_pair_t<8>(a, grid, s); return true;
    case 9: *err = load_pair_t<9>(a, grid, s); return true;
    case 10: *err = load_pair_t<10>(a, grid, s); return true;
    case 11: *err = load_pair_t<11>(a, grid, s); return true;
    case 12: *err = load_pair_t<12>(a, grid, s); return true;
    default: return false;
  }
}

bool launch_row_c2r_spec(int P, const RowArgs& a, dim3 grid, cudaStream_t s, cudaError_t* err) {
  switch (spec_ln(P, a.M, a.C, 128, 2048)) {
    case 7: *err = row_c2r_t<7>(a, grid, s); return true;
    case 8: *err = row_c2r_t<8>(a, grid, s); return true;
    case 9: *err = row_c2r_t<9>(a, grid, s); return true;
    case 10: *err = row_c2r_t<10>(a, grid, s); return true;
    case 11: *err = row_c2r_t<11>(a, grid, s); return true;
    default: return false;
  }
}

}  // namespace grf
