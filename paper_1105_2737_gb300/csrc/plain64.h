// Plain FP64 form (plain64.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace grf {

struct Plain64Geom {
  int d;
  int n[3];
};

// One field: writes N_tot doubles to `out`.  bufA/bufB hold N_tot complex doubles each.
// stab: FP64 folded s_K table; tw: FP64 twiddles tw[L + k] = exp(2 pi i k / L).
// twax[i]: exp(2 pi i k / N_i), k < N_i, for an axis whose size is not a power
// of two (its radix-3/5/7 stages read it); may be NULL for the other axes.
cudaError_t plain64_field(const Plain64Geom& g, int alg, uint64_t key, const double* stab, const double2* tw,
                          const double2* const* twax, double2* bufA, double2* bufB, double* out, cudaStream_t s);
// The same steps in FP32 (FP32 plans on grids that are not powers of two), with
// the fused path's FP32 noise: stab the FP32 folded table, tw the FP32
// twiddles, trig = exp(2 pi i h / 256) for Box-Muller.
cudaError_t plain32_field(const Plain64Geom& g, int alg, uint64_t key, const float* stab, const float2* tw,
                          const float2* const* twax, const float2* trig, float2* bufA, float2* bufB, float* out,
                          cudaStream_t s);
// twn[k] = exp(2 pi i k / n), k < n (FP64-computed; rounded for the FP32 form).
cudaError_t build_axis_twiddles(double2* twn, int n, cudaStream_t s);
cudaError_t build_axis_twiddles(float2* twn, int n, cudaStream_t s);

}  // namespace grf
