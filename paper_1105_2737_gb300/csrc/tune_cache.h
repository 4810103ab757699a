// Tuning cache shared by the plan tuner (api.cu) and the batch tuner
// (batch.cu): lines "key v1 v2 ..." in a text file, the last line of a key
// wins.  Path: GRF_TUNE_CACHE, else $HOME/.cache/grf_gb300_tune.txt.
#pragma once
#include <string>
#include <vector>

namespace grf {

std::string tune_gpu_name();
bool tune_cache_lookup(const std::string& key, std::vector<int>* values);
void tune_cache_store(const std::string& key, const std::vector<int>& values);

}  // namespace grf
