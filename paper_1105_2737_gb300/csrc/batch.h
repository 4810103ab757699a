// Uneven batches: many fields of different shapes and dimensions, sampled by
// per-shape launches in one graph or by one persistent kernel (batch.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include "grf.h"

namespace grf {

struct BatchPlan;

grf_status batch_plan_build(BatchPlan** out, int64_t count, const int* d, const int64_t* n, const double* L,
                            const grf_spectrum* spec, std::string* err);
grf_status batch_plan_sample(BatchPlan* b, uint64_t seed, void* const* out, cudaStream_t s, int* status,
                             bool use_graph, std::string* err);
int64_t batch_plan_total_points(const BatchPlan* b);
grf_status batch_plan_debug(BatchPlan* b, int withhold_field, double timeout_ms);
// 0: per-shape launches (default), 1: one persistent kernel.
grf_status batch_plan_set_mode(BatchPlan* b, int mode);
int batch_plan_mode(const BatchPlan* b);
void batch_plan_free(BatchPlan* b);

}  // namespace grf
