#include "batch.h"

namespace grf {

struct BatchPlan {
  int64_t count = 0;
  int64_t total_points = 0;
};

grf_status batch_plan_build(BatchPlan** out, int64_t, const int*, const int64_t*, const double*,
                            const grf_spectrum*, std::string* err) {
  *out = nullptr;
  *err = "uneven batches are not built yet";
  return GRF_ERR_UNSUPPORTED;
}

grf_status batch_plan_sample(BatchPlan*, uint64_t, void* const*, cudaStream_t, int*, bool, std::string* err) {
  *err = "uneven batches are not built yet";
  return GRF_ERR_UNSUPPORTED;
}

int64_t batch_plan_total_points(const BatchPlan* b) { return b ? b->total_points : 0; }
void batch_plan_free(BatchPlan* b) { delete b; }

}  // namespace grf
