// The four-step stages of long 1-D Algorithm 2 fields (the paired first stage
// and the second stage) compiled for fixed geometries: transform length
// 2^LN = 64 .. 2048 with 4096 / 2^LN columns per CTA, 256 threads of 16 points
// (see pass_kernels.cuh).
#include "pass_kernels.cuh"

namespace grf {

namespace {

template <int LN>
cudaError_t fourstep_spec_t(int stage, const FourStepArgs& a, int64_t nfields, cudaStream_t s) {
  constexpr int CC = 4096 >> LN;
  const size_t smem = col_smem_bytes(1 << LN, CC);
  if (stage == 3) {  // the paired first stage: CC / 2 mirror pairs of columns per CTA
    constexpr int H = CC / 2;
    static_assert(H >= 1, "paired stage with at least two columns per CTA");
    auto k = fourstep_stage1_pair<16, LN, CC>;
    cudaError_t e = prepare_kernel((const void*)k, 256, smem);
    if (e != cudaSuccess) return e;
    k<<<dim3((unsigned)((a.A / 2 + 1 + H - 1) / H), 1, (unsigned)nfields), 256, smem, s>>>(a);
  } else {
    auto k = fourstep_stage2<16, LN, CC>;
    cudaError_t e = prepare_kernel((const void*)k, 256, smem);
    if (e != cudaSuccess) return e;
    k<<<dim3((unsigned)(a.B / CC), 1, (unsigned)nfields), 256, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace

bool launch_fourstep_spec(int stage, const FourStepArgs& a, int64_t nfields, cudaStream_t s, cudaError_t* err) {
  if (stage != 2 && stage != 3) return false;
  const int len = stage == 2 ? a.A : a.B;
  const int ln = stage == 2 ? a.logA : a.logB;
  if (ln < 6 || ln > 11 || (1 << ln) != len || a.C != (4096 >> ln)) return false;
  switch (ln) {
    case 6: *err = fourstep_spec_t<6>(stage, a, nfields, s); return true;
    case 7: *err = fourstep_spec_t<7>(stage, a, nfields, s); return true;
    case 8: *err = fourstep_spec_t<8>(stage, a, nfields, s); return true;
    case 9: *err = fourstep_spec_t<9>(stage, a, nfields, s); return true;
    case 10: *err = fourstep_spec_t<10>(stage, a, nfields, s); return true;
    case 11: *err = fourstep_spec_t<11>(stage, a, nfields, s); return true;
    default: return false;
  }
}

}  // namespace grf
