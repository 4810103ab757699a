#include "tune_cache.h"

#include <cuda_runtime.h>
#include <sys/stat.h>

#include <cstdlib>
#include <fstream>
#include <mutex>
#include <sstream>

namespace grf {
namespace {

std::mutex g_mu;

std::string cache_path() {
  const char* e = std::getenv("GRF_TUNE_CACHE");
  if (e && *e) return e;
  const char* h = std::getenv("HOME");
  return std::string(h ? h : "/tmp") + "/.cache/grf_gb300_tune.txt";
}

}  // namespace

std::string tune_gpu_name() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "unknown";
  std::string s = pr.name;
  for (char& c : s)
    if (c == ' ' || c == '\n' || c == '\t') c = '_';
  return s;
}

bool tune_cache_lookup(const std::string& key, std::vector<int>* values) {
  std::lock_guard<std::mutex> lock(g_mu);
  std::ifstream f(cache_path());
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string k;
    if (!(is >> k) || k != key) continue;
    std::vector<int> v;
    int x;
    while (is >> x) v.push_back(x);
    *values = v;
    found = true;
  }
  return found;
}

void tune_cache_store(const std::string& key, const std::vector<int>& values) {
  std::lock_guard<std::mutex> lock(g_mu);
  const std::string path = cache_path();
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos) mkdir(path.substr(0, slash).c_str(), 0755);  // best effort
  std::ofstream f(path, std::ios::app);
  if (!f) return;
  f << key;
  for (int v : values) f << " " << v;
  f << "\n";
}

}  // namespace grf
