// A 2-D sampling entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they want a
// field: code that runs inside a host application which owns the device's
// memory (a fixed pool handed out by its own allocator, with raw cudaMalloc
// forbidden), and latency-critical loops where cudaMalloc / cudaFree would
// implicitly synchronise the device.  grf_sample_2d_static serves them: its
// tables and its intermediate half spectrum live in one file-scope device
// array, `g_noalloc_scratch`, that the CUDA driver reserves when it loads this
// library on a device and keeps until the process exits.  The caller passes
// only the output.
//
// The array is shared by every call on a device and keeps the last call's
// contents; every call rebuilds what it reads before reading it.  Calls that
// overlap on the GPU (several streams, or several host threads) race on the
// array: keep calls of this entry point on one stream at a time.
#include <algorithm>
#include <mutex>

#include "grf.h"
#include "kernels.h"

namespace grf {

// Largest grid: N1, N2 <= 1024.  Worst-case use, each part rounded up to 256
// bytes as the call lays them out: twiddles and stage tables for length 1024,
// (2 * 1024 + kStageTableEntries) complex floats (about 112 KiB); the folded
// s_K table, 513 x 513 floats (about 1.0 MiB); one field's half spectrum,
// 1024 x 513 complex floats (about 4.0 MiB).  About 5.1 MiB in all.
constexpr int kNoAllocMaxSide = 1024;
constexpr size_t kNoAllocScratchBytes = 6u << 20;
constexpr size_t round256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kNoAllocWorstBytes =
    round256((size_t)(2 * kNoAllocMaxSide + kStageTableEntries) * 8) +
    round256((size_t)(kNoAllocMaxSide / 2 + 1) * (kNoAllocMaxSide / 2 + 1) * 4) +
    (size_t)kNoAllocMaxSide * (kNoAllocMaxSide / 2 + 1) * 8;
static_assert(kNoAllocWorstBytes <= kNoAllocScratchBytes, "the largest grid must fit the scratch array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

void set_last_error(const char* msg);  // api.cu

namespace {

std::mutex g_mu;
void* g_scratch_addr[64] = {nullptr};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
int lg2(int64_t x) {
  int r = 0;
  while ((int64_t(1) << r) < x) ++r;
  return r;
}

grf_status reject(grf_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

// Columns per CTA for the axis-1 pass and rows per CTA for the c2r pass:
// 256 threads, at most 64 KiB of shared memory, no more columns than exist.
int cols_per_cta(int N, int64_t ncols) {
  const int P = points_per_thread(N);
  int C = 256 / (N / P);
  if (C < 1) C = 1;
  while (C > 1 && col_smem_bytes(N, C) > 64 * 1024) C >>= 1;
  while (C > 1 && C / 2 >= ncols) C >>= 1;
  return C;
}
int rows_per_cta(int M, int64_t nrows) {
  const int P = M >= 16 ? 16 : M;
  int C = 256 / (M / P);
  if (C < 1) C = 1;
  while (C > 1 && row_smem_bytes(M, C) > 64 * 1024) C >>= 1;
  while (C > 1 && C / 2 >= nrows) C >>= 1;
  return C;
}

}  // namespace
}  // namespace grf

using namespace grf;

extern "C" grf_status grf_sample_2d_static(const int64_t* n, const double* L, const grf_spectrum* spec,
                                           uint64_t seed, int64_t batch, float* out, void* stream) {
  if (!n || !L || !spec || !out) return reject(GRF_ERR_INVALID_ARG, "grf_sample_2d_static: NULL pointer");
  if (batch < 1) return reject(GRF_ERR_INVALID_ARG, "grf_sample_2d_static: batch must be >= 1");
  for (int i = 0; i < 2; ++i) {
    if (n[i] < 2 || (n[i] & 1)) return reject(GRF_ERR_INVALID_ARG, "grf_sample_2d_static: N_i must be even and >= 2");
    if (!pow2(n[i])) return reject(GRF_ERR_UNSUPPORTED, "grf_sample_2d_static: N_i must be a power of two");
    if (n[i] > kNoAllocMaxSide)
      return reject(GRF_ERR_INVALID_ARG,
                    "grf_sample_2d_static: N_i above 1024, the size of the fixed scratch array; use grf_sample");
    if (!(L[i] > 0)) return reject(GRF_ERR_INVALID_ARG, "grf_sample_2d_static: L_i must be > 0");
  }
  if (spec->family < 0 || spec->family > 2 || !(spec->sigma > 0))
    return reject(GRF_ERR_INVALID_ARG, "grf_sample_2d_static: bad spectrum");
  if (spec->family <= 1 && !(spec->ell > 0)) return reject(GRF_ERR_INVALID_ARG, "grf_sample_2d_static: ell must be > 0");
  if (spec->family == 0 && !(spec->nu > 0)) return reject(GRF_ERR_INVALID_ARG, "grf_sample_2d_static: nu must be > 0");
  if (spec->family == 2 && (!(spec->m > 0) || spec->k < 1 || spec->l < 1 || spec->n < 1))
    return reject(GRF_ERR_INVALID_ARG, "grf_sample_2d_static: bad paper-family parameters");
  if (spec->normalize_discrete)
    return reject(GRF_ERR_UNSUPPORTED, "grf_sample_2d_static: normalize_discrete needs grf_plan_create");

  // Set-up, once per device with that device current: the device address of the
  // scratch array (host code cannot use the symbol itself as a device pointer).
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return reject(GRF_ERR_CUDA, "grf_sample_2d_static: no current CUDA device");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return reject(GRF_ERR_CUDA, "grf_sample_2d_static: cudaGetSymbolAddress failed");
      g_scratch_addr[dev] = p;
    }
    base = (unsigned char*)g_scratch_addr[dev];
  }

  const int N1 = (int)n[0], N2 = (int)n[1], M = N2 / 2;
  const int maxlen = std::max(256, std::max(N1, N2));  // length 256: Box-Muller's coarse angles
  const size_t tw_bytes = align256((size_t)(2 * maxlen + kStageTableEntries) * sizeof(float2));
  const size_t fold = (size_t)(N1 / 2 + 1) * (M + 1);
  const size_t st_bytes = align256(fold * sizeof(float));
  const size_t ws_bytes = (size_t)N1 * (M + 1) * sizeof(float2);
  if (tw_bytes + st_bytes + ws_bytes > kNoAllocScratchBytes)
    return reject(GRF_ERR_INVALID_ARG, "grf_sample_2d_static: grid does not fit the fixed scratch array");
  float2* tw = (float2*)base;
  float* stab = (float*)(base + tw_bytes);
  float2* ws = (float2*)(base + tw_bytes + st_bytes);
  cudaStream_t s = (cudaStream_t)stream;

  // Tables (rebuilt on every call: the array keeps whatever the last call left).
  SpecParams sp{};
  sp.family = spec->family;
  sp.sigma = spec->sigma;
  sp.ell = spec->ell;
  sp.nu = spec->nu;
  sp.m = spec->m;
  sp.k = spec->k;
  sp.l = spec->l;
  sp.n = spec->n;
  sp.scale = 1.0;
  sp.d = 2;
  sp.L[0] = L[0];
  sp.L[1] = L[1];
  sp.L[2] = 1.0;
  sp.nn[0] = N1;
  sp.nn[1] = N2;
  sp.nn[2] = 1;
  if (build_twiddles(tw, maxlen, s) != cudaSuccess || build_stab(stab, nullptr, sp, 0.0, s) != cudaSuccess)
    return reject(GRF_ERR_CUDA, "grf_sample_2d_static: table build failed");

  HalfGeom g{};
  g.d = 2;
  g.N1 = N1;
  g.Nmid = 1;
  g.M = M;
  g.Q = (uint32_t)(M / 2 + 1);
  g.seed = seed;
  g.stab = stab;
  g.trig = tw + 256;
  ColArgs a{};
  a.N = N1;
  a.logN = lg2(N1);
  a.C = cols_per_cta(N1, M / 2 + 1);
  a.ncols = M + 1;
  a.zpair = 1;  // pairs of columns (p, M - p): the pass writes Z of the c2r split
  a.twz = tw + N2;
  a.T = 1;
  a.logT = 0;
  a.bstride = (int64_t)N1 * (M + 1);
  a.out = ws;
  a.tw = tw + N1;
  a.tws = tw + 2 * maxlen;
  RowArgs r{};
  r.M = M;
  r.logM = lg2(M);
  r.C = rows_per_cta(M, N1);
  r.rows_per_field = N1;
  r.nrows = N1;
  r.T = 1;
  r.logT = 0;
  r.inH = ws;
  r.twM = tw + M;
  r.twN = tw + 2 * M;
  r.tws = tw + 2 * maxlen;
  const dim3 gc((unsigned)((M / 2 + 1 + a.C - 1) / a.C), 1, 1);
  const dim3 gr((unsigned)((r.nrows + r.C - 1) / r.C));
  // One field at a time through the one-field half-spectrum slot; the stream
  // orders the reuse of the slot between consecutive fields.
  for (int64_t b = 0; b < batch; ++b) {
    a.g = g;
    a.g.field0 = b;
    r.g = a.g;
    r.outR = out + b * (int64_t)N1 * N2;
    if (launch_col(COL_NOISE, COL_INV, points_per_thread(N1), a, gc, s) != cudaSuccess ||
        launch_row(ROW_LOAD_Z, ROW_C2R, M >= 16 ? 16 : M, r, gr, s) != cudaSuccess)
      return reject(GRF_ERR_CUDA, "grf_sample_2d_static: kernel launch failed");
  }
  return GRF_OK;
}
