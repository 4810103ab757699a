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
cudaError_t plain64_field(const Plain64Geom& g, int alg, uint64_t key, const double* stab, const double2* tw,
                          double2* bufA, double2* bufB, double* out, cudaStream_t s);

}  // namespace grf
