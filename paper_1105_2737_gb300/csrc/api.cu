// C ABI of the GRF library: plan creation (validation, FP64 table builds,
// workspace, schedules), sampling (Algorithm 2 and Algorithm 1 of §3),
// the adjoint with respect to (sigma, ell, nu), and the forward r2c DFT.
#include "grf.h"
#include "kernels.h"
#include "plain64.h"
#include "batch.h"
#include "tune_cache.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace grf;

namespace {

thread_local std::string g_last_error;

grf_status fail(grf_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

grf_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? GRF_ERR_OOM : GRF_ERR_CUDA;
}

#define GRF_CUDA(call, where)                      \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
bool smooth_2357(int64_t x) {
  if (x < 1) return false;
  for (int p : {2, 3, 5, 7})
    while (x % p == 0) x /= p;
  return x == 1;
}
int ilog2(int64_t x) {
  int r = 0;
  while ((int64_t(1) << r) < x) ++r;
  return r;
}
int64_t next_pow2(int64_t x) {
  int64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// psi(x): recurrence up to x >= 10, then the asymptotic series
// (Abramowitz & Stegun 6.3.5, 6.3.18).
double digamma_host(double x) {
  double acc = 0.0;
  while (x < 10.0) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  const double x2 = 1.0 / (x * x);
  const double series =
      x2 * (1.0 / 12 - x2 * (1.0 / 120 - x2 * (1.0 / 252 - x2 * (1.0 / 240 - x2 * (1.0 / 132)))));
  return acc + std::log(x) - 0.5 / x - series;
}

struct ColSched {
  int C = 1, P = 16;
};
struct RowSched {
  int C = 1, P = 16;
};

const size_t kSmemCap = 100 * 1024;

ColSched choose_col(int N, int64_t ncols, int max_threads = 256) {
  ColSched s;
  s.P = points_per_thread(N);
  const int TPT = N / s.P;
  int C = max_threads / TPT;
  if (C < 1) C = 1;
  while (C > 1 && col_smem_bytes(N, C) > kSmemCap) C >>= 1;
  const int64_t cp = next_pow2(ncols);
  if (C > cp) C = (int)cp;
  s.C = C;
  return s;
}

RowSched choose_row(int M, int64_t nrows, int max_threads = 256) {
  RowSched s;
  s.P = M >= 16 ? 16 : M;
  const int TPT = M / s.P;
  int C = max_threads / TPT;
  if (C < 1) C = 1;
  while (C > 1 && row_smem_bytes(M, C) > kSmemCap) C >>= 1;
  const int64_t rp = next_pow2(nrows);
  if (C > rp) C = (int)rp;
  s.C = C;
  return s;
}

int max_threads_for(int P) { return P >= 16 ? 256 : (P == 8 ? 512 : 1024); }

// Schedules the tuner tries for transforms of length N over `ncols` columns
// (or rows): radix P in {16, 8, 4} (P = N for the tiniest lengths), and every
// power-of-two count of columns per CTA that fits the radix's thread limit.
std::vector<ColSched> schedule_candidates(int N, int64_t ncols, bool rows) {
  std::vector<ColSched> out;
  for (int P : {16, 8, 4, 2, 1}) {
    if (P > N || (P < 4 && P != N)) continue;
    const int TPT = N / P;
    const int maxC = max_threads_for(P) / TPT;
    for (int C = 1; C <= maxC && C <= next_pow2(ncols); C *= 2) {
      const size_t smem = rows ? row_smem_bytes(N, C) : col_smem_bytes(N, C);
      if (smem > kSmemCap) break;
      ColSched cs;
      cs.P = P;
      cs.C = C;
      out.push_back(cs);
    }
  }
  return out;
}

}  // namespace

struct grf_plan_s {
  int kind = 0;  // 0: one shape; 1: uneven batch
  int d = 0;
  int64_t n[3] = {1, 1, 1};
  double L[3] = {1, 1, 1};
  grf_spectrum spec{};
  int alg = 2, prec = 0;
  int64_t max_batch = 1;
  int device = 0;
  double norm_scale = 1.0;

  // geometry
  int N1 = 1, Nmid = 1, M = 1;
  int64_t ntot = 0, hsize = 0, fold_size = 0;

  // FP32 tables and workspace
  float2* tw = nullptr;
  int twmax = 0;
  float* stab = nullptr;
  float* stabT = nullptr;  // 1-D four-step: s_k laid out along k2 (build_stab_fourstep)
  float* dstab = nullptr;
  float2* ws = nullptr;
  int64_t chunk = 1;
  double* partial = nullptr;
  int64_t partial_cap = 0;
  int T = 1;  // 2-D tile of the half-spectrum workspace
  ColSched colA, colB;
  RowSched row;
  // four-step 1-D (M > 4096): M = A * B
  int fsA = 0, fsB = 0, fsC1 = 1, fsC2 = 1;
  // 2-D / 3-D pipelining: the batch in `pipe` chunks, first passes on the
  // caller's stream, the others on tail_stream
  int pipe = 1;
  int row_tma = 0;  // c2r pass: 0 = row kernel, 1 = persistent kernel fed by bulk async copies
  int plane_R = 0;  // 3-D: the plane path's axis-2 split N2 = R Q (0: the three-pass form)
  int64_t ws_field = 0;  // workspace entries per field
  bool sched_cached = false;  // the schedule came from the tuning cache at creation
  int gs_ctas = 1;  // grid-stride CTAs per SM of each pass when pipelined (0: full grids)
  int num_sms = 0;
  cudaStream_t tail_stream = nullptr;
  cudaEvent_t pipe_ev[9] = {};

  // FP64 plain form
  double2* tw64 = nullptr;
  double* stab64 = nullptr;
  double2* bufA = nullptr;
  double2* bufB = nullptr;
  // FP32 plans on grids that are not powers of two take the plain form in FP32
  bool mixed = false;
  float2* buf32A = nullptr;
  float2* buf32B = nullptr;
  // per-axis twiddles exp(2 pi i k / N_i) of the plain form's radix-3/5/7 stages
  // (axes whose size is not a power of two; NULL otherwise)
  double2* twax64[3] = {nullptr, nullptr, nullptr};
  float2* twax32[3] = {nullptr, nullptr, nullptr};
  // FP32 2-D Algorithm 2 plans of those sizes: the fused passes of mixed_fused.cu
  bool mixfused = false;
  int mixC1 = 1, mixlogT = 0, mixthreads2 = 256;
  int mixnst[2] = {0, 0};
  int mixrad[2][16] = {};
  float2* mixtab[2] = {nullptr, nullptr};  // stage tables of N1 and M

  // host delivery
  static constexpr int kCopyStreams = 4;
  cudaStream_t copy_stream = nullptr;
  cudaStream_t copy_streams[kCopyStreams] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_part[2][kCopyStreams] = {};
  cudaEvent_t ev_done[2] = {nullptr, nullptr};
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  void* stage[2] = {nullptr, nullptr};
  int64_t stage_fields = 0;

  int* status = nullptr;  // device status word

  // 1-D covariance estimator (grf_cov_origin): one chunk of fields and its partial sums
  float* cov_buf = nullptr;
  double* cov_partial = nullptr;

  BatchPlan* batch = nullptr;

  // Neumann / Dirichlet fields (kind 2): n[] holds the intervals N_i, a field
  // has prod (N_i + 1) points; t_K in field layout
  int bc = 0;
  float* bctab = nullptr;
  int bcC[3] = {1, 1, 1};  // sequences per CTA of the pass along each axis

  // per-launch timing
  std::vector<cudaEvent_t> tev;
  std::vector<int> tkind;
  int64_t tcap = 0, tused = 0;
};

namespace {

void free_plan(grf_plan p) {
  if (!p) return;
  cudaFree(p->tw);
  cudaFree(p->stab);
  cudaFree(p->stabT);
  cudaFree(p->bctab);
  cudaFree(p->dstab);
  cudaFree(p->ws);
  cudaFree(p->partial);
  cudaFree(p->tw64);
  cudaFree(p->stab64);
  cudaFree(p->bufA);
  cudaFree(p->bufB);
  cudaFree(p->buf32A);
  cudaFree(p->buf32B);
  for (int i = 0; i < 3; ++i) {
    cudaFree(p->twax64[i]);
    cudaFree(p->twax32[i]);
  }
  cudaFree(p->mixtab[0]);
  cudaFree(p->mixtab[1]);
  for (int i = 0; i < 2; ++i) {
    cudaFree(p->stage[i]);
    if (p->ev_done[i]) cudaEventDestroy(p->ev_done[i]);
    if (p->ev_copied[i]) cudaEventDestroy(p->ev_copied[i]);
  }
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  if (p->tail_stream) cudaStreamDestroy(p->tail_stream);
  for (cudaEvent_t e : p->pipe_ev)
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < grf_plan_s::kCopyStreams; ++i) {
    if (p->copy_streams[i]) cudaStreamDestroy(p->copy_streams[i]);
    for (int j = 0; j < 2; ++j)
      if (p->ev_part[j][i]) cudaEventDestroy(p->ev_part[j][i]);
  }
  cudaFree(p->status);
  cudaFree(p->cov_buf);
  cudaFree(p->cov_partial);
  if (p->batch) batch_plan_free(p->batch);
  for (cudaEvent_t e : p->tev) cudaEventDestroy(e);
  delete p;
}

template <class T>
cudaError_t dmalloc(T** ptr, size_t count) {
  if (count == 0) count = 1;
  return cudaMalloc((void**)ptr, count * sizeof(T));
}

grf_status validate_spec(const grf_spectrum* spec) {
  if (!spec) return fail(GRF_ERR_INVALID_ARG, "spec is NULL");
  if (spec->family < 0 || spec->family > 2) return fail(GRF_ERR_INVALID_ARG, "unknown spectral family");
  if (!(spec->sigma > 0) || !std::isfinite(spec->sigma)) return fail(GRF_ERR_INVALID_ARG, "sigma must be > 0");
  if (spec->family <= 1 && (!(spec->ell > 0) || !std::isfinite(spec->ell)))
    return fail(GRF_ERR_INVALID_ARG, "ell must be > 0");
  if (spec->family == 0 && (!(spec->nu > 0) || !std::isfinite(spec->nu)))
    return fail(GRF_ERR_INVALID_ARG, "nu must be > 0");
  if (spec->family == 2 && (!(spec->m > 0) || spec->k < 1 || spec->l < 1 || spec->n < 1))
    return fail(GRF_ERR_INVALID_ARG, "paper family needs m > 0 and k, l, n >= 1");
  return GRF_OK;
}

SpecParams spec_params(const grf_plan_s* p) {
  SpecParams sp{};
  sp.family = p->spec.family;
  sp.sigma = p->spec.sigma;
  sp.ell = p->spec.ell;
  sp.nu = p->spec.nu;
  sp.m = p->spec.m;
  sp.k = p->spec.k;
  sp.l = p->spec.l;
  sp.n = p->spec.n;
  sp.scale = p->norm_scale;
  sp.d = p->d;
  for (int i = 0; i < 3; ++i) {
    sp.L[i] = p->L[i];
    sp.nn[i] = (int)p->n[i];
  }
  return sp;
}

// sum_K S(p_K)/|D| over the full grid, in FP64 on the host (folded, with multiplicities).
double discrete_sum(const grf_plan_s* p) {
  const double PI = 3.141592653589793238462643383279502884;
  const int d = p->d;
  const grf_spectrum& s = p->spec;
  double vol = 1.0;
  for (int i = 0; i < d; ++i) vol *= p->L[i];
  double c = 0.0;
  if (s.family == 0)
    c = std::pow(2.0 * std::sqrt(PI) * s.ell, d) * std::exp(std::lgamma(s.nu + 0.5 * d) - std::lgamma(s.nu));
  else if (s.family == 1)
    c = std::pow(2.0 * PI * s.ell * s.ell, 0.5 * d);
  int64_t F[3] = {1, 1, 1};
  for (int i = 0; i < d; ++i) F[i] = p->n[i] / 2 + 1;
  double total = 0.0;
  for (int64_t a = 0; a < F[0]; ++a)
    for (int64_t b = 0; b < F[1]; ++b)
      for (int64_t e = 0; e < F[2]; ++e) {
        const int64_t f[3] = {a, b, e};
        double p2 = 0.0, mult = 1.0, s2k = 0.0;
        for (int i = 0; i < d; ++i) {
          const double pi = (double)f[i] / p->L[i];
          p2 += pi * pi;
          if (s.family == 2) s2k += std::pow(pi, 2.0 * s.k);
          if (f[i] != 0 && f[i] != p->n[i] / 2) mult *= 2.0;
        }
        double S;
        if (s.family == 0) S = s.sigma * s.sigma * c * std::pow(1.0 + s.ell * s.ell * 4 * PI * PI * p2, -s.nu - 0.5 * d);
        else if (s.family == 1) S = s.sigma * s.sigma * c * std::exp(-2 * PI * PI * s.ell * s.ell * p2);
        else S = s.sigma * s.sigma * std::pow(std::pow(s.m, (double)(s.k * s.l)) + std::pow(s2k, (double)s.l), -(double)s.n);
        total += mult * S / vol;
      }
  return total;
}

grf_status ensure_partial(grf_plan p, int64_t count) {
  if (count <= p->partial_cap) return GRF_OK;
  cudaFree(p->partial);
  p->partial = nullptr;
  p->partial_cap = 0;
  GRF_CUDA(dmalloc(&p->partial, (size_t)count * 3), "partial buffer");
  p->partial_cap = count;
  return GRF_OK;
}

HalfGeom half_geom(const grf_plan_s* p, uint64_t seed, int64_t field0) {
  HalfGeom g{};
  g.d = p->d;
  g.N1 = p->N1;
  g.Nmid = p->Nmid;
  g.M = p->M;
  g.Q = (uint32_t)(p->M / 2 + 1);
  g.seed = seed;
  g.field0 = field0;
  g.stab = p->stab;
  g.dstab = p->dstab;
  g.inv_sigma = (float)(1.0 / p->spec.sigma);
  g.trig = p->tw + 256;
  g.alg1_scale = (float)(1.0 / std::sqrt((double)p->ntot));
  return g;
}

const float2* twp(const grf_plan_s* p, int len) { return p->tw + len; }

// Radices of a length n = 2^a 3^b 5^c 7^e for the mixed-radix stages: the odd
// ones first (the first stage writes at a stride of its radix, which an odd
// radix spreads over all shared-memory banks), then 8s and a 4 or a 2 for the
// rest of the powers of two.  False if n has another factor or needs more
// than 16 stages.
bool mixed_radices(int n, int* rad, int* nst) {
  int k = 0;
  auto push = [&](int r) {
    if (k < 16) rad[k] = r;
    ++k;
  };
  for (int r : {3, 5, 7})
    while (n % r == 0) push(r), n /= r;
  while (n % 8 == 0) push(8), n /= 8;
  if (n % 4 == 0) push(4), n /= 4;
  if (n % 2 == 0) push(2), n /= 2;
  *nst = k;
  return n == 1 && k >= 1 && k <= 16;
}

// The schedule of the fused mixed-radix passes: C1 columns per CTA of pass 1
// (C1 N1 <= 4096 entries, 16 B each in two buffers); pass 2 takes T = 2^logT
// rows per CTA, the largest T <= 4 dividing N1 whose tile fits in 48 KB (four
// CTAs of 256 threads per SM; measured at 3000^2, 1000^2 and 3000 x 4096 against
// the neighbouring T and 512 threads).  GRF_MIXED_T and GRF_MIXED_THREADS
// override T and the threads of pass 2.
bool mixed_schedule(int N1, int M, int* C1, int* logT, int* threads2, int (*rad)[16], int* nst) {
  if (N1 > 4096 || M > 4096 || N1 < 2 || M < 2) return false;
  if (!mixed_radices(N1, rad[0], &nst[0]) || !mixed_radices(M, rad[1], &nst[1])) return false;
  int c = 4096 / N1;
  if (c > M + 1) c = M + 1;
  *C1 = c < 1 ? 1 : c;
  int t = 4;
  if (const char* te = std::getenv("GRF_MIXED_T")) t = std::max(1, std::min(8, std::atoi(te)));
  const bool forced = std::getenv("GRF_MIXED_T") != nullptr;
  while (t > 1 && (N1 % t || (t & (t - 1)) || mixed_c2r_smem_bytes(M, t) > (forced ? 200 : 48) * 1024 + 64)) t >>= 1;
  *logT = t == 8 ? 3 : t == 4 ? 2 : t == 2 ? 1 : 0;
  *threads2 = 256;
  if (const char* th = std::getenv("GRF_MIXED_THREADS")) *threads2 = std::atoi(th) == 512 ? 512 : 256;
  return true;
}

MixedArgs mixed_args(const grf_plan_s* p, uint64_t seed, float* out) {
  MixedArgs a{};
  a.N1 = p->N1;
  a.M = p->M;
  a.logT = p->mixlogT;
  a.threads2 = p->mixthreads2;
  a.C1 = p->mixC1;
  a.nst1 = p->mixnst[0];
  a.nst2 = p->mixnst[1];
  for (int i = 0; i < 16; ++i) {
    a.rad1[i] = p->mixrad[0][i];
    a.rad2[i] = p->mixrad[1][i];
  }
  a.st1 = p->mixtab[0];
  a.st2 = p->mixtab[1];
  a.tw2 = p->twax32[1] ? p->twax32[1] : twp(p, 2 * p->M);
  a.g = half_geom(p, seed, 0);
  a.ws = p->ws;
  a.ws_stride = p->ws_field;
  a.out = out;
  return a;
}

// Column pass along axis 1 (the transform length N1); plane = whole field.
ColArgs col_axis1(const grf_plan_s* p, const HalfGeom& g, const float2* in, float2* out, int T) {
  ColArgs a{};
  a.N = p->N1;
  a.logN = ilog2(p->N1);
  a.C = p->colA.C;
  a.ncols = (int64_t)p->Nmid * (p->M + 1);
  a.T = T;
  a.logT = ilog2(T);
  a.ostride = 0;
  a.bstride = p->hsize;
  a.in = in;
  a.out = out;
  a.tw = twp(p, p->N1);
  a.tws = p->tw + 2 * p->twmax;
  a.plane_is_k1 = 1;
  a.g = g;
  return a;
}

// Column pass along axis 2 of a 3-D half spectrum (planes = j1 or k1).
ColArgs col_axis2(const grf_plan_s* p, const HalfGeom& g, const float2* in, float2* out) {
  ColArgs a{};
  a.N = p->Nmid;
  a.logN = ilog2(p->Nmid);
  a.C = p->colB.C;
  a.ncols = p->M + 1;
  a.T = 1;
  a.logT = 0;
  a.ostride = (int64_t)p->Nmid * (p->M + 1);
  a.bstride = p->hsize;
  a.in = in;
  a.out = out;
  a.tw = twp(p, p->Nmid);
  a.tws = p->tw + 2 * p->twmax;
  a.plane_is_k1 = 0;
  a.g = g;
  return a;
}

RowArgs row_args(const grf_plan_s* p, const HalfGeom& g, int64_t nfields, int T) {
  RowArgs r{};
  r.M = p->M;
  r.logM = ilog2(p->M);
  r.C = p->row.C;
  r.rows_per_field = p->ntot / p->n[p->d - 1];
  r.nrows = nfields * r.rows_per_field;
  r.T = T;
  r.logT = ilog2(T);
  r.twM = twp(p, p->M);
  r.twN = twp(p, 2 * p->M);
  r.tws = p->tw + 2 * p->twmax;
  r.g = g;
  return r;
}

// Pair mode for the last column pass of a plane of M + 1 columns: it writes Z
// of the c2r split (see col_body), which the c2r pass reads.
ColArgs zpair(const grf_plan_s* p, ColArgs a) {
  a.zpair = 1;
  a.twz = twp(p, 2 * p->M);
  return a;
}

dim3 col_grid(const ColArgs& a, int64_t planes, int64_t nfields) {
  const int64_t slots = a.zpair ? a.g.M / 2 + 1 : a.ncols;
  return dim3((unsigned)((slots + a.C - 1) / a.C), (unsigned)planes, (unsigned)nfields);
}
dim3 row_grid(const RowArgs& r) { return dim3((unsigned)((r.nrows + r.C - 1) / r.C)); }

#define LAUNCH(call, where)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, where);      \
  } while (0)

// Cache key of a plan's schedule: the GPU, the grid and the algorithm.
std::string plan_key(const grf_plan_s* p) {
  std::string k = "plan|" + tune_gpu_name() + "|" + std::to_string(p->d);
  for (int i = 0; i < 3; ++i) k += "x" + std::to_string(p->n[i]);
  k += "|alg" + std::to_string(p->alg) + "|b" + std::to_string(p->max_batch);
  return k;
}

bool valid_sched(const ColSched& c, int N, int64_t ncols, bool rows) {
  for (const ColSched& x : schedule_candidates(N, ncols, rows))
    if (x.P == c.P && x.C == c.C) return true;
  return false;
}

// Values: T, colA.P, colA.C, colB.P, colB.C, row.P, row.C, pipe, row_tma
// (absent: 0).  Applied only if every entry is a schedule this plan could have
// chosen itself.
bool apply_schedule(grf_plan_s* p, const std::vector<int>& v) {
  if ((v.size() != 8 && v.size() != 9) || p->d < 2) return false;
  const int tma = v.size() == 9 ? v[8] : 0;
  if (tma < 0 || tma > 1) return false;
  ColSched a, b, r;
  a.P = v[1];
  a.C = v[2];
  b.P = v[3];
  b.C = v[4];
  r.P = v[5];
  r.C = v[6];
  const int T = v[0];
  if (T < 1 || (T & (T - 1)) || p->N1 % T || (p->d == 3 && T != 1)) return false;
  if (!valid_sched(a, p->N1, (int64_t)p->Nmid * (p->M + 1), false)) return false;
  if (p->d == 3 && !valid_sched(b, p->Nmid, p->M + 1, false)) return false;
  if (!valid_sched(r, p->M, p->max_batch * (p->ntot / p->n[p->d - 1]), true)) return false;
  if (v[7] < 1 || v[7] > 8) return false;
  p->T = T;
  p->colA = a;
  if (p->d == 3) p->colB = b;
  p->row.P = r.P;
  p->row.C = r.C;
  p->pipe = v[7];
  p->row_tma = tma;
  return true;
}

// A launch bracketed by timing events when the plan records them.
#define TLAUNCH(kind, call, where)                                                   \
  do {                                                                               \
    const bool t_ = p->tused < p->tcap;                                              \
    if (t_) cudaEventRecord(p->tev[2 * p->tused], s);                                \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, where);                              \
    if (t_) {                                                                        \
      cudaEventRecord(p->tev[2 * p->tused + 1], s);                                  \
      p->tkind[p->tused] = (kind);                                                   \
    }                                                                                \
    if (p->tcap > 0) ++p->tused;                                                     \
  } while (0)

// FP32 sampling of fields [f0, f0 + nb) into out (already offset to field f0),
// through the half-spectrum workspace `ws` (nb fields).  In 2-D and 3-D the
// first pass (noise + axis 1) runs on `s` and the remaining passes on `st`,
// which waits for it: with st != s, the first pass of the next chunk overlaps
// the last passes of this one.
grf_status sample_chunk_fp32(grf_plan p, uint64_t seed, int64_t f0, int64_t nb, float* out, cudaStream_t s,
                             float2* ws = nullptr, cudaStream_t st = nullptr, cudaEvent_t ev = nullptr) {
  const HalfGeom g = half_geom(p, seed, f0);
  if (!ws) ws = p->ws;
  if (p->d == 1 && p->M > 4096) {
    FourStepArgs f{};
    f.A = p->fsA;
    f.logA = ilog2(p->fsA);
    f.B = p->fsB;
    f.logB = ilog2(p->fsB);
    f.M = p->M;
    f.N = 2 * p->M;
    f.T = p->fsC1 / 2;  // stage 1 takes fsC1 / 2 mirror pairs of columns per CTA
    f.logT = ilog2(p->fsC1 / 2);
    f.Y = p->ws;
    f.Yin = p->ws;
    f.out = out;
    f.twA = twp(p, p->fsA);
    f.twB = twp(p, p->fsB);
    f.twM = twp(p, p->M);
    f.twN = twp(p, 2 * p->M);
    f.tws = p->tw + 2 * p->twmax;
    f.stab = p->stab;
    f.stabT = p->stabT;
    f.tw2B = twp(p, 2 * p->fsB);
    f.twMA = twp(p, p->fsA);
    f.trig = p->tw + 256;
    f.seed = seed;
    f.field0 = f0;
    f.C = p->fsC1;
    TLAUNCH(GRF_KERNEL_ROWS_1D, launch_fourstep(3, 16, f, nb, s), "four-step stage 1");
    f.C = p->fsC2;
    TLAUNCH(GRF_KERNEL_ROWS_1D, launch_fourstep(2, 16, f, nb, s), "four-step stage 2");
    return GRF_OK;
  }
  if (p->d == 1) {
    RowArgs r = row_args(p, g, nb, 1);
    r.outR = out;
    if (p->alg == 2) TLAUNCH(GRF_KERNEL_ROWS_1D, launch_row(ROW_NOISE_H, ROW_C2R, p->row.P, r, row_grid(r), s), "1-D c2r");
    else TLAUNCH(GRF_KERNEL_ROWS_1D, launch_row(ROW_NOISE_REAL, ROW_R2C_SCALE_C2R, p->row.P, r, row_grid(r), s), "1-D alg1");
    return GRF_OK;
  }
  if (p->d == 3 && p->alg == 2 && p->plane_R) {
    // the plane path: noise + axis 1 + the first radix-R step of axis 2, then
    // one CTA per sub-plane for the rest of axis 2 and the c2r pass
    PlaneArgs pl{};
    pl.N1 = p->N1;
    pl.N2 = p->Nmid;
    pl.M = p->M;
    pl.R = p->plane_R;
    pl.Q = p->Nmid / p->plane_R;
    pl.S3 = p->M + 2;
    pl.ws = ws;
    pl.out = out;
    pl.tw = p->tw;
    pl.tws = p->tw + 2 * p->twmax;
    pl.status = p->status;
    ColArgs a = col_axis1(p, g, nullptr, ws, 1);
    if (p->N1 >= 256) {
      TLAUNCH(GRF_KERNEL_NOISE_COLUMNS, launch_plane3_noise(a, pl, nb, s), "3-D plane pass 1");
    } else {  // the column pass, whole planes with padded rows
      a.pitch3 = pl.S3;
      a.bstride = (int64_t)p->N1 * p->Nmid * pl.S3;
      TLAUNCH(GRF_KERNEL_NOISE_COLUMNS, launch_col(COL_NOISE, COL_INV, p->colA.P, a, col_grid(a, 1, nb), s),
              "3-D plane pass 1");
    }
    if (st && st != s) {
      GRF_CUDA(cudaEventRecord(ev, s), "pipeline event");
      GRF_CUDA(cudaStreamWaitEvent(st, ev, 0), "pipeline wait");
      s = st;
    }
    TLAUNCH(GRF_KERNEL_ROWS_C2R, launch_plane3_c2r(pl, nb, s), "3-D plane pass 2");
    return GRF_OK;
  }
  const int T = p->d == 2 ? p->T : 1;
  const bool gs = st && st != s && p->gs_ctas > 0;
  if (p->alg == 2) {
    ColArgs a = col_axis1(p, g, nullptr, ws, T);
    if (p->d == 2) a = zpair(p, a);
    if (gs)
      TLAUNCH(GRF_KERNEL_NOISE_COLUMNS, launch_col_noise_gs(p->colA.P, a, col_grid(a, 1, nb), p->gs_ctas * p->num_sms, s),
              "noise + axis-1 pass");
    else
      TLAUNCH(GRF_KERNEL_NOISE_COLUMNS, launch_col(COL_NOISE, COL_INV, p->colA.P, a, col_grid(a, 1, nb), s),
              "noise + axis-1 pass");
  } else {
    RowArgs r = row_args(p, g, nb, T);
    r.outH = ws;
    TLAUNCH(GRF_KERNEL_ROWS_R2C, launch_row(ROW_NOISE_REAL, ROW_R2C, p->row.P, r, row_grid(r), s), "alg1 noise + r2c");
    if (p->d == 3) {
      ColArgs b = col_axis2(p, g, ws, ws);
      TLAUNCH(GRF_KERNEL_COLUMNS, launch_col(COL_LOAD, COL_FWD, p->colB.P, b, col_grid(b, p->N1, nb), s), "alg1 axis-2 forward");
    }
    ColArgs a = col_axis1(p, g, ws, ws, T);
    if (p->d == 2) a = zpair(p, a);
    TLAUNCH(GRF_KERNEL_COLUMNS, launch_col(COL_LOAD, COL_FWD_SCALE_INV, p->colA.P, a, col_grid(a, 1, nb), s), "alg1 axis-1 scale");
  }
  if (st && st != s) {
    GRF_CUDA(cudaEventRecord(ev, s), "pipeline event");
    GRF_CUDA(cudaStreamWaitEvent(st, ev, 0), "pipeline wait");
    s = st;
  }
  if (p->d == 3) {
    ColArgs b = zpair(p, col_axis2(p, g, ws, ws));
    TLAUNCH(GRF_KERNEL_COLUMNS, launch_col(COL_LOAD, COL_INV, p->colB.P, b, col_grid(b, p->N1, nb), s), "axis-2 inverse");
  }
  RowArgs r = row_args(p, g, nb, T);
  r.inH = ws;
  r.outR = out;
  if (p->row_tma && c2r_tma_ok(r))
    TLAUNCH(GRF_KERNEL_ROWS_C2R, launch_row_c2r_tma(p->row.P, r, gs ? p->gs_ctas : 0, p->num_sms, p->status, s),
            "c2r pass (bulk copies)");
  else if (gs)
    TLAUNCH(GRF_KERNEL_ROWS_C2R, launch_row_c2r_gs(p->row.P, r, row_grid(r).x, p->gs_ctas * p->num_sms, s),
            "c2r pass");
  else
    TLAUNCH(GRF_KERNEL_ROWS_C2R, launch_row(ROW_LOAD_Z, ROW_C2R, p->row.P, r, row_grid(r), s), "c2r pass");
  return GRF_OK;
}

grf_status check_plan(grf_plan p) {
  if (!p) return fail(GRF_ERR_INVALID_ARG, "plan is NULL");
  return GRF_OK;
}

}  // namespace

namespace grf {
// Error text for entry points defined in other translation units.
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace grf

namespace {

// Neumann / Dirichlet fields: the noise + last-axis launch, then one in-place
// launch per remaining axis, from the last but one to the first.
grf_status sample_bc(grf_plan p, uint64_t seed, int64_t batch, float* out, cudaStream_t s) {
  if (!out) return fail(GRF_ERR_INVALID_ARG, "out is NULL");
  if (batch < 1 || batch > p->max_batch) return fail(GRF_ERR_INVALID_ARG, "batch must be in [1, max_batch]");
  const int d = p->d;
  int64_t pts[3] = {1, 1, 1};
  for (int i = 0; i < d; ++i) pts[i] = p->n[i] + 1;
  for (int ax = d - 1; ax >= 0; --ax) {
    R2rArgs a{};
    a.f = out;
    a.field_stride = p->ntot;
    a.lines_per_field = p->ntot / pts[ax];
    a.nlines = batch * a.lines_per_field;
    a.inner = 1;
    for (int i = ax + 1; i < d; ++i) a.inner *= pts[i];
    a.N = (int)p->n[ax];
    a.logNF = ilog2(2 * p->n[ax]);
    a.C = p->bcC[ax];
    a.logC = ilog2(a.C);
    a.logG = a.logC + 1;
    a.bc = p->bc;
    a.d = d;
    a.axis = ax;
    for (int i = 0; i < 3; ++i) a.pts[i] = pts[i];
    a.noise = ax == d - 1;
    a.tab = p->bctab;
    a.seed = seed;
    a.field0 = 0;
    a.tw = p->tw + 2 * p->n[ax];
    a.tws = p->tw + 2 * p->twmax;
    a.trig = p->tw + 256;
    TLAUNCH(a.noise ? GRF_KERNEL_R2R_NOISE : GRF_KERNEL_R2R, launch_r2r(a, s),
            a.noise ? "boundary field: noise + last axis" : "boundary field: axis pass");
  }
  return GRF_OK;
}

}  // namespace

extern "C" {

grf_status grf_bc_plan_create(grf_plan* out, int d, const int64_t* n, const double* L, const grf_spectrum* spec,
                              int bc, int64_t max_batch) {
  g_last_error.clear();
  if (!out) return fail(GRF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (d < 1 || d > 3) return fail(GRF_ERR_INVALID_ARG, "d must be 1, 2 or 3");
  if (!n || !L) return fail(GRF_ERR_INVALID_ARG, "n or L is NULL");
  grf_status st = validate_spec(spec);
  if (st != GRF_OK) return st;
  if (bc != GRF_BC_NEUMANN && bc != GRF_BC_DIRICHLET) return fail(GRF_ERR_INVALID_ARG, "bc must be 1 or 2");
  if (max_batch < 1 || max_batch > 65535) return fail(GRF_ERR_INVALID_ARG, "max_batch must be in [1, 65535]");
  for (int i = 0; i < d; ++i) {
    if (n[i] < 2) return fail(GRF_ERR_INVALID_ARG, "every N_i must be >= 2");
    if (!(L[i] > 0) || !std::isfinite(L[i])) return fail(GRF_ERR_INVALID_ARG, "every L_i must be > 0");
  }
  if (spec->normalize_discrete) return fail(GRF_ERR_UNSUPPORTED, "normalize_discrete is for periodic plans");
  int64_t ntot = 1;
  for (int i = 0; i < d; ++i) {
    if (!is_pow2(n[i]) || n[i] > 4096) return fail(GRF_ERR_UNSUPPORTED, "N_i must be a power of two <= 4096");
    ntot *= n[i] + 1;
  }
  grf_plan p = new (std::nothrow) grf_plan_s();
  if (!p) return fail(GRF_ERR_OOM, "host allocation");
  p->kind = 2;
  p->d = d;
  for (int i = 0; i < d; ++i) {
    p->n[i] = n[i];
    p->L[i] = L[i];
  }
  p->spec = *spec;
  p->prec = GRF_FP32;
  p->max_batch = max_batch;
  p->bc = bc;
  p->ntot = ntot;
  p->chunk = max_batch;  // host delivery: fields per staged chunk at most
  cudaGetDevice(&p->device);
  int64_t maxlen = 256;  // the length-256 table also serves Box-Muller's coarse angles
  for (int i = 0; i < d; ++i) maxlen = std::max<int64_t>(maxlen, 2 * n[i]);
  p->twmax = (int)maxlen;
  for (int i = 0; i < d; ++i) p->bcC[i] = r2r_lines_per_cta((int)n[i]);
  cudaError_t e;
  if ((e = dmalloc(&p->status, 1)) != cudaSuccess || (e = cudaMemset(p->status, 0, sizeof(int))) != cudaSuccess ||
      (e = dmalloc(&p->tw, 2 * maxlen + kStageTableEntries)) != cudaSuccess ||
      (e = build_twiddles(p->tw, (int)maxlen, nullptr)) != cudaSuccess || (e = dmalloc(&p->bctab, ntot)) != cudaSuccess ||
      (e = build_bc_table(p->bctab, spec_params(p), bc, nullptr)) != cudaSuccess ||
      (e = cudaStreamSynchronize(nullptr)) != cudaSuccess) {
    grf_status r = cuda_fail(e, "boundary plan tables");
    free_plan(p);
    return r;
  }
  *out = p;
  return GRF_OK;
}


const char* grf_status_string(grf_status s) {
  switch (s) {
    case GRF_OK: return "ok";
    case GRF_ERR_INVALID_ARG: return "invalid argument";
    case GRF_ERR_UNSUPPORTED: return "unsupported configuration";
    case GRF_ERR_OOM: return "out of device memory";
    case GRF_ERR_CUDA: return "CUDA error";
    case GRF_ERR_TIMEOUT: return "device wait timed out";
    case GRF_ERR_NOT_HERMITIAN: return "input is not Hermitian";
    default: return "unknown status";
  }
}

const char* grf_last_error(void) { return g_last_error.c_str(); }

grf_status grf_plan_create(grf_plan* out, int d, const int64_t* n, const double* L, const grf_spectrum* spec,
                           int alg, int prec, int64_t max_batch) {
  g_last_error.clear();
  if (!out) return fail(GRF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (d < 1 || d > 3) return fail(GRF_ERR_INVALID_ARG, "d must be 1, 2 or 3");
  if (!n || !L) return fail(GRF_ERR_INVALID_ARG, "n or L is NULL");
  grf_status st = validate_spec(spec);
  if (st != GRF_OK) return st;
  if (alg != GRF_ALG_ONE_FFT && alg != GRF_ALG_TWO_FFT) return fail(GRF_ERR_INVALID_ARG, "alg must be 1 or 2");
  if (prec != GRF_FP32 && prec != GRF_FP64) return fail(GRF_ERR_INVALID_ARG, "prec must be 0 or 1");
  if (max_batch < 1 || max_batch > 65535) return fail(GRF_ERR_INVALID_ARG, "max_batch must be in [1, 65535]");
  for (int i = 0; i < d; ++i) {
    if (n[i] < 2 || (n[i] & 1)) return fail(GRF_ERR_INVALID_ARG, "every N_i must be even and >= 2");
    if (!(L[i] > 0) || !std::isfinite(L[i])) return fail(GRF_ERR_INVALID_ARG, "every L_i must be > 0");
  }
  // powers of two take the fused FP32 kernels; other sizes 2^a 3^b 5^c 7^e the
  // plain form (radix 2, 3, 5 and 7 stages), in FP64 or FP32
  bool all_pow2 = true;
  for (int i = 0; i < d; ++i) {
    if (!smooth_2357(n[i])) return fail(GRF_ERR_UNSUPPORTED, "N_i must be 2^a 3^b 5^c 7^e");
    all_pow2 = all_pow2 && is_pow2(n[i]);
  }
  const bool mixed = prec == GRF_FP32 && !all_pow2;
  for (int i = 0; i < d; ++i) {
    int64_t lim = (i < d - 1) ? 4096 : 8192;
    if (d == 1 && (prec == GRF_FP64 || alg == GRF_ALG_ONE_FFT || mixed)) lim = int64_t(1) << 22;  // four-step c2r
    if (n[i] > lim) return fail(GRF_ERR_UNSUPPORTED, "grid size above the supported maximum");
  }

  grf_plan p = new (std::nothrow) grf_plan_s();
  if (!p) return fail(GRF_ERR_OOM, "host allocation");
  p->d = d;
  for (int i = 0; i < d; ++i) {
    p->n[i] = n[i];
    p->L[i] = L[i];
  }
  p->spec = *spec;
  p->alg = alg;
  p->prec = prec;
  p->max_batch = max_batch;
  p->mixed = mixed;
  cudaGetDevice(&p->device);
  p->M = (int)(n[d - 1] / 2);
  p->N1 = d >= 2 ? (int)n[0] : 1;
  p->Nmid = d == 3 ? (int)n[1] : 1;
  p->ntot = 1;
  for (int i = 0; i < d; ++i) p->ntot *= n[i];
  p->hsize = (int64_t)p->N1 * p->Nmid * (p->M + 1);
  p->fold_size = (int64_t)(p->N1 / 2 + 1) * (p->Nmid / 2 + 1) * (p->M + 1);
  if (spec->normalize_discrete) {
    const double tot = discrete_sum(p);
    p->norm_scale = spec->sigma * spec->sigma / tot;
  }

  int64_t maxlen = 256;  // the length-256 table also serves Box-Muller's coarse angles
  for (int i = 0; i < d; ++i) maxlen = maxlen > n[i] ? maxlen : n[i];
  while (!is_pow2(maxlen)) ++maxlen;  // the tables hold powers of two up to maxlen
  p->twmax = (int)maxlen;
  cudaStream_t s = nullptr;
  const SpecParams sp = spec_params(p);
  cudaError_t e;
#define PLAN_CUDA(call, where)                 \
  do {                                         \
    e = (call);                                \
    if (e != cudaSuccess) {                    \
      grf_status r_ = cuda_fail(e, where);     \
      free_plan(p);                            \
      return r_;                               \
    }                                          \
  } while (0)

  PLAN_CUDA(dmalloc(&p->status, 1), "status word");
  PLAN_CUDA(cudaMemset(p->status, 0, sizeof(int)), "status word");
  if (mixed) {
    PLAN_CUDA(dmalloc(&p->tw, 2 * maxlen + kStageTableEntries), "twiddle table");
    PLAN_CUDA(build_twiddles(p->tw, (int)maxlen, s), "twiddle build");
    PLAN_CUDA(dmalloc(&p->stab, p->fold_size), "s table");
    PLAN_CUDA(build_stab(p->stab, nullptr, sp, 0.0, s), "s table build");
    for (int i = 0; i < d; ++i)
      if (!is_pow2(n[i])) {
        PLAN_CUDA(dmalloc(&p->twax32[i], n[i]), "axis twiddles");
        PLAN_CUDA(build_axis_twiddles(p->twax32[i], (int)n[i], s), "axis twiddles");
      }
    p->chunk = max_batch;
    const char* mf = std::getenv("GRF_MIXED_FUSED");  // "0": keep the plain form
    p->mixfused = d == 2 && alg == GRF_ALG_ONE_FFT && !(mf && mf[0] == '0') &&
                  mixed_schedule(p->N1, p->M, &p->mixC1, &p->mixlogT, &p->mixthreads2, p->mixrad, p->mixnst);
    if (p->mixfused) {
      for (int i = 0; i < 2; ++i) {
        PLAN_CUDA(dmalloc(&p->mixtab[i], i == 0 ? p->N1 : p->M), "stage table");
        PLAN_CUDA(build_mixed_stage_table(p->mixtab[i], p->mixrad[i], p->mixnst[i], s), "stage table");
      }
      p->ws_field = p->hsize;
      PLAN_CUDA(dmalloc(&p->ws, (size_t)(p->chunk * p->ws_field)), "workspace");
    } else {
      PLAN_CUDA(dmalloc(&p->buf32A, p->ntot), "FP32 plain buffer");
      PLAN_CUDA(dmalloc(&p->buf32B, p->ntot), "FP32 plain buffer");
    }
  } else if (prec == GRF_FP32) {
    PLAN_CUDA(dmalloc(&p->tw, 2 * maxlen + kStageTableEntries), "twiddle table");
    PLAN_CUDA(build_twiddles(p->tw, (int)maxlen, s), "twiddle build");
    PLAN_CUDA(dmalloc(&p->stab, p->fold_size), "s table");
    const bool grad = spec->family <= 1 && !spec->normalize_discrete;
    double dig = 0.0;
    if (grad) {
      PLAN_CUDA(dmalloc(&p->dstab, 2 * p->fold_size), "ds table");
      if (spec->family == 0) dig = digamma_host(spec->nu + 0.5 * d) - digamma_host(spec->nu);
    }
    PLAN_CUDA(build_stab(p->stab, p->dstab, sp, dig, s), "s table build");
    // schedules
    if (d == 1 && p->M > 4096) {
      const int lm = ilog2(p->M);
      p->fsB = 1 << ((lm + 1) / 2);
      p->fsA = p->M / p->fsB;
      p->fsC1 = 4096 / p->fsB;  // 256 threads of 16 points
      if (p->fsC1 > p->fsA) p->fsC1 = p->fsA;
      p->fsC2 = 4096 / p->fsA;
      if (p->fsC2 > p->fsB) p->fsC2 = p->fsB;
      p->chunk = max_batch;
      PLAN_CUDA(dmalloc(&p->ws, (size_t)(p->chunk * p->M)), "four-step workspace");
      PLAN_CUDA(dmalloc(&p->stabT, (size_t)p->M), "four-step s table");
      PLAN_CUDA(build_stab_fourstep(p->stabT, p->stab, p->fsA, p->fsB, s), "four-step s table build");
    } else if (d == 1) {
      p->row = choose_row(p->M, max_batch);
    } else {
      p->colA = choose_col(p->N1, (int64_t)p->Nmid * (p->M + 1));
      if (d == 3) p->colB = choose_col(p->Nmid, p->M + 1);
      p->row = choose_row(p->M, max_batch * (p->ntot / n[d - 1]));
      p->T = 1;
      if (d == 2 && p->N1 >= 256) {
        p->T = 8;
        while (p->T > 1 && p->N1 % p->T) p->T >>= 1;
      }
      p->chunk = max_batch;
      p->ws_field = p->hsize;
      if (d == 3 && alg == GRF_ALG_ONE_FFT) {
        const char* pe3 = std::getenv("GRF_PLANE3");  // "0": keep the three-pass form
        if (!(pe3 && pe3[0] == '0')) p->plane_R = plane3_radix(p->N1, p->Nmid, p->M);
        if (p->plane_R)
          p->ws_field = std::max<int64_t>(p->hsize, (int64_t)plane3_ws_entries(p->N1, p->Nmid, p->M));
      }
      PLAN_CUDA(dmalloc(&p->ws, (size_t)(p->chunk * p->ws_field)), "workspace");
      {  // a tuned schedule for this GPU and problem, if one was stored
        std::vector<int> v;
        if (tune_cache_lookup(plan_key(p), &v)) p->sched_cached = apply_schedule(p, v);
      }
      if (const char* pe = std::getenv("GRF_PIPELINE")) p->pipe = std::max(1, std::min(8, std::atoi(pe)));
      if (const char* ge = std::getenv("GRF_GS_CTAS")) p->gs_ctas = std::max(0, std::min(8, std::atoi(ge)));
      cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    }
  } else {
    PLAN_CUDA(dmalloc(&p->tw64, 2 * maxlen), "FP64 twiddle table");
    PLAN_CUDA(build_twiddles_d(p->tw64, (int)maxlen, s), "FP64 twiddle build");
    PLAN_CUDA(dmalloc(&p->stab64, p->fold_size), "FP64 s table");
    PLAN_CUDA(build_stab_d(p->stab64, sp, s), "FP64 s table build");
    PLAN_CUDA(dmalloc(&p->bufA, p->ntot), "FP64 buffer");
    PLAN_CUDA(dmalloc(&p->bufB, p->ntot), "FP64 buffer");
    for (int i = 0; i < d; ++i)
      if (!is_pow2(n[i])) {
        PLAN_CUDA(dmalloc(&p->twax64[i], n[i]), "axis twiddles");
        PLAN_CUDA(build_axis_twiddles(p->twax64[i], (int)n[i], s), "axis twiddles");
      }
  }
  PLAN_CUDA(cudaStreamSynchronize(s), "plan table build");
#undef PLAN_CUDA
  *out = p;
  if (const char* te = std::getenv("GRF_TUNE"))
    if (te[0] == '1' && prec == GRF_FP32 && d >= 2) grf_plan_tune(p, nullptr);
  return GRF_OK;
}

grf_status grf_plan_set_spectrum(grf_plan p, const grf_spectrum* spec, void* stream) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (p->kind == 1) return fail(GRF_ERR_INVALID_ARG, "batch plans keep their spectra");
  st = validate_spec(spec);
  if (st != GRF_OK) return st;
  if (spec->family != p->spec.family || (spec->normalize_discrete != 0) != (p->spec.normalize_discrete != 0))
    return fail(GRF_ERR_INVALID_ARG, "the family and normalisation mode are fixed at plan creation");
  cudaStream_t s = (cudaStream_t)stream;
  if (p->kind == 2) {  // boundary fields: the c_K table
    p->spec = *spec;
    LAUNCH(build_bc_table(p->bctab, spec_params(p), p->bc, s), "boundary c_K table build");
    return GRF_OK;
  }
  p->spec = *spec;
  p->norm_scale = spec->normalize_discrete ? spec->sigma * spec->sigma / discrete_sum(p) : 1.0;
  const SpecParams sp = spec_params(p);
  if (p->prec == GRF_FP32) {
    double dig = 0.0;
    if (spec->family == 0) dig = digamma_host(spec->nu + 0.5 * p->d) - digamma_host(spec->nu);
    LAUNCH(build_stab(p->stab, p->dstab, sp, dig, s), "s table build");
    if (p->stabT) LAUNCH(build_stab_fourstep(p->stabT, p->stab, p->fsA, p->fsB, s), "four-step s table build");
  } else {
    LAUNCH(build_stab_d(p->stab64, sp, s), "FP64 s table build");
  }
  return GRF_OK;
}

grf_status grf_sample(grf_plan p, uint64_t seed, int64_t batch, void* out, void* stream) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (p->kind == 2) return sample_bc(p, seed, batch, (float*)out, (cudaStream_t)stream);
  if (p->kind != 0) return fail(GRF_ERR_INVALID_ARG, "batch plans use grf_batch_sample");
  if (!out) return fail(GRF_ERR_INVALID_ARG, "out is NULL");
  if (batch < 1 || batch > p->max_batch) return fail(GRF_ERR_INVALID_ARG, "batch must be in [1, max_batch]");
  cudaStream_t s = (cudaStream_t)stream;
  if (p->mixfused) {
    const MixedArgs a = mixed_args(p, seed, (float*)out);
    TLAUNCH(GRF_KERNEL_NOISE_COLUMNS, launch_mixed_noise(a, batch, s), "mixed-radix noise pass");
    TLAUNCH(GRF_KERNEL_ROWS_C2R, launch_mixed_c2r(a, batch, s), "mixed-radix c2r pass");
    return GRF_OK;
  }
  if (p->prec == GRF_FP64 || p->mixed) {
    Plain64Geom g{};
    g.d = p->d;
    for (int i = 0; i < 3; ++i) g.n[i] = (int)p->n[i];
    for (int64_t b = 0; b < batch; ++b) {
      if (p->mixed)
        TLAUNCH(GRF_KERNEL_PLAIN64,
                plain32_field(g, p->alg, seed + (uint64_t)b, p->stab, p->tw, p->twax32, p->tw + 256, p->buf32A,
                              p->buf32B, (float*)out + b * p->ntot, s),
                "FP32 plain field");
      else
        TLAUNCH(GRF_KERNEL_PLAIN64,
                plain64_field(g, p->alg, seed + (uint64_t)b, p->stab64, p->tw64, p->twax64, p->bufA, p->bufB,
                              (double*)out + b * p->ntot, s),
                "FP64 plain field");
    }
    return GRF_OK;
  }
  if (p->d >= 2 && p->pipe > 1 && batch > 1) {
    // pipeline: chunk k's noise + axis-1 pass (ALU-bound) on s overlaps chunk
    // k-1's c2r pass (memory-bound) on the tail stream
    if (!p->tail_stream) {
      GRF_CUDA(cudaStreamCreateWithFlags(&p->tail_stream, cudaStreamNonBlocking), "tail stream");
      for (cudaEvent_t& e : p->pipe_ev) GRF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    }
    const int K = (int)(batch < p->pipe ? batch : p->pipe);
    const int64_t per = (batch + K - 1) / K;
    GRF_CUDA(cudaEventRecord(p->pipe_ev[8], s), "pipeline fork");
    GRF_CUDA(cudaStreamWaitEvent(p->tail_stream, p->pipe_ev[8], 0), "pipeline fork");
    int k = 0;
    for (int64_t f0 = 0; f0 < batch; f0 += per, ++k) {
      const int64_t nb = batch - f0 < per ? batch - f0 : per;
      st = sample_chunk_fp32(p, seed, f0, nb, (float*)out + f0 * p->ntot, s, p->ws + f0 * p->ws_field, p->tail_stream,
                             p->pipe_ev[k % 8]);
      if (st != GRF_OK) return st;
    }
    GRF_CUDA(cudaEventRecord(p->pipe_ev[8], p->tail_stream), "pipeline join");
    GRF_CUDA(cudaStreamWaitEvent(s, p->pipe_ev[8], 0), "pipeline join");
    return GRF_OK;
  }
  const int64_t chunk = (p->d == 1 && p->M <= 4096) ? batch : p->chunk;
  for (int64_t f0 = 0; f0 < batch; f0 += chunk) {
    const int64_t nb = batch - f0 < chunk ? batch - f0 : chunk;
    st = sample_chunk_fp32(p, seed, f0, nb, (float*)out + f0 * p->ntot, s);
    if (st != GRF_OK) return st;
  }
  return GRF_OK;
}

grf_status grf_plan_tune(grf_plan p, void* stream) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (p->kind != 0 || p->prec != GRF_FP32 || p->d < 2 || p->mixed)
    return fail(GRF_ERR_UNSUPPORTED, "the tuner covers FP32 2-D and 3-D plans on powers of two");
  const char* force = std::getenv("GRF_TUNE_FORCE");
  if (p->sched_cached && !(force && force[0] == '1')) return GRF_OK;  // already tuned on this GPU
  if (p->plane_R) return GRF_OK;  // the 3-D plane path has one schedule
  cudaStream_t s = (cudaStream_t)stream;
  // enough fields for a few waves of CTAs, within max_batch
  int64_t bt = (int64_t)((64ll << 20) / p->ntot);
  bt = std::max<int64_t>(1, std::min<int64_t>(bt, p->max_batch));
  float* out = nullptr;
  GRF_CUDA(cudaMalloc(&out, (size_t)bt * p->ntot * sizeof(float)), "tuning output");
  const int64_t old_cap = p->tcap;
  // mean time per launch kind over two timed calls (after one warm-up call)
  auto measure = [&](double* ms_kind) -> grf_status {
    for (int k = 0; k < 8; ++k) ms_kind[k] = 0.0;
    grf_status r = grf_sample(p, 1, bt, out, stream);
    if (r != GRF_OK) return r;
    GRF_CUDA(cudaStreamSynchronize(s), "tuning sync");
    r = grf_plan_timing(p, 64);
    if (r != GRF_OK) return r;
    for (int i = 0; i < 2 && r == GRF_OK; ++i) r = grf_sample(p, 2 + i, bt, out, stream);
    if (r != GRF_OK) return r;
    int kinds[64];
    float ms[64];
    const int64_t n = grf_plan_timing_read(p, kinds, ms, 64);
    for (int64_t i = 0; i < n && i < 64; ++i)
      if (kinds[i] >= 0 && kinds[i] < 8) ms_kind[kinds[i]] += ms[i] / 2.0;
    return GRF_OK;
  };
  const int64_t ncolA = (int64_t)p->Nmid * (p->M + 1);
  const int64_t nrows = p->max_batch * (p->ntot / p->n[p->d - 1]);
  std::vector<int> tvals = {1};
  if (p->d == 2)
    for (int T = 2; T <= 16; T *= 2)
      if (p->N1 % T == 0) tvals.push_back(T);
  double best_total = 1e30;
  std::vector<int> best;
  double ms[8];
  for (int T : tvals) {
    p->T = T;
    double total = 0.0;
    ColSched ba = p->colA;
    double bta = 1e30;
    for (const ColSched& c : schedule_candidates(p->N1, ncolA, false)) {
      p->colA = c;
      if ((st = measure(ms)) != GRF_OK) break;
      if (ms[GRF_KERNEL_NOISE_COLUMNS] < bta) {
        bta = ms[GRF_KERNEL_NOISE_COLUMNS];
        ba = c;
      }
    }
    if (st != GRF_OK) break;
    p->colA = ba;
    total += bta;
    if (p->d == 3) {
      ColSched bb = p->colB;
      double btb = 1e30;
      for (const ColSched& c : schedule_candidates(p->Nmid, p->M + 1, false)) {
        p->colB = c;
        if ((st = measure(ms)) != GRF_OK) break;
        if (ms[GRF_KERNEL_COLUMNS] < btb) {
          btb = ms[GRF_KERNEL_COLUMNS];
          bb = c;
        }
      }
      if (st != GRF_OK) break;
      p->colB = bb;
      total += btb;
    }
    ColSched br;
    br.P = p->row.P;
    br.C = p->row.C;
    int btma = 0;
    double btr = 1e30;
    for (const ColSched& c : schedule_candidates(p->M, nrows, true)) {
      p->row.P = c.P;
      p->row.C = c.C;
      for (int tma = 0; tma <= 1 && st == GRF_OK; ++tma) {
        if (tma) {  // only where the tuning batch takes the bulk-copy kernel
          RowArgs r = row_args(p, half_geom(p, 0, 0), bt, p->d == 2 ? T : 1);
          r.inH = p->ws;
          if (!c2r_tma_ok(r)) continue;
        }
        p->row_tma = tma;
        if ((st = measure(ms)) != GRF_OK) break;
        if (ms[GRF_KERNEL_ROWS_C2R] < btr) {
          btr = ms[GRF_KERNEL_ROWS_C2R];
          br = c;
          btma = tma;
        }
      }
      if (st != GRF_OK) break;
    }
    if (st != GRF_OK) break;
    p->row.P = br.P;
    p->row.C = br.C;
    p->row_tma = btma;
    total += btr;
    if (total < best_total) {
      best_total = total;
      best = {T, p->colA.P, p->colA.C, p->colB.P, p->colB.C, p->row.P, p->row.C, 1, btma};
    }
  }
  if (st == GRF_OK && !best.empty()) {
    apply_schedule(p, best);
    // pipelining depth, timed on whole calls
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float bestp = 1e30f;
    int pipe_best = 1;
    for (int pp : {1, 2, 4}) {
      p->pipe = pp;
      grf_sample(p, 1, bt, out, stream);
      cudaEventRecord(e0, s);
      for (int i = 0; i < 2; ++i) grf_sample(p, 2 + i, bt, out, stream);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float t = 1e30f;
      cudaEventElapsedTime(&t, e0, e1);
      if (t < bestp * 0.98f) {
        bestp = t;
        pipe_best = pp;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    best[7] = pipe_best;
    apply_schedule(p, best);
    tune_cache_store(plan_key(p), best);
  }
  grf_plan_timing(p, old_cap > 0 ? old_cap : 0);
  cudaFree(out);
  return st;
}

grf_status grf_sample_host(grf_plan p, uint64_t seed, int64_t batch, void* host_out, void* stream) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (p->kind == 1) return fail(GRF_ERR_INVALID_ARG, "batch plans use grf_batch_sample");
  if (!host_out) return fail(GRF_ERR_INVALID_ARG, "host_out is NULL");
  if (batch < 1 || batch > p->max_batch) return fail(GRF_ERR_INVALID_ARG, "batch must be in [1, max_batch]");
  cudaStream_t s = (cudaStream_t)stream;
  // Pinned host memory that is mapped into the device's address space is
  // written by the kernels directly (on Grace-Blackwell over NVLink-C2C): on
  // GB300 a steady 160 GiB/s, where the staged copies below reach 175 GiB/s in
  // some runs and half of that in others.  Only for plans whose kernels write
  // each output once with ordinary stores (not the boundary fields, which
  // transform the output in place, nor the passes that store by bulk copies).
  // GRF_HOST_DIRECT=0 keeps the staged copies; other host memory always takes them.
  cudaPointerAttributes attr;
  const char* direct = std::getenv("GRF_HOST_DIRECT");
  const bool plain_stores = p->kind == 0 && !(p->d == 3 && p->plane_R) && !p->row_tma;
  if (plain_stores && !(direct && direct[0] == '0') && cudaPointerGetAttributes(&attr, host_out) == cudaSuccess &&
      attr.type == cudaMemoryTypeHost && attr.devicePointer != nullptr) {
    st = grf_sample(p, seed, batch, attr.devicePointer, stream);
    if (st != GRF_OK) return st;
    GRF_CUDA(cudaStreamSynchronize(s), "host delivery sync");
    return GRF_OK;
  }
  cudaGetLastError();  // clear a failed attribute query on unregistered memory
  const size_t esz = p->prec == GRF_FP64 ? sizeof(double) : sizeof(float);
  const size_t field_bytes = (size_t)p->ntot * esz;
  int64_t per = (int64_t)((64u << 20) / field_bytes);
  if (per < 1) per = 1;
  if (p->prec == GRF_FP32 && (p->d > 1 || p->M > 4096) && per > p->chunk) per = p->chunk;
  if (per > batch) per = batch;
  if (p->stage_fields < per) {
    for (int i = 0; i < 2; ++i) {
      cudaFree(p->stage[i]);
      p->stage[i] = nullptr;
    }
    p->stage_fields = 0;
    for (int i = 0; i < 2; ++i) GRF_CUDA(cudaMalloc(&p->stage[i], per * field_bytes), "host staging buffer");
    p->stage_fields = per;
  }
  if (!p->copy_stream) {
    GRF_CUDA(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking), "copy stream");
    for (int i = 0; i < 2; ++i) {
      GRF_CUDA(cudaEventCreateWithFlags(&p->ev_done[i], cudaEventDisableTiming), "event");
      GRF_CUDA(cudaEventCreateWithFlags(&p->ev_copied[i], cudaEventDisableTiming), "event");
    }
    for (int i = 0; i < grf_plan_s::kCopyStreams; ++i) {
      GRF_CUDA(cudaStreamCreateWithFlags(&p->copy_streams[i], cudaStreamNonBlocking), "copy stream");
      for (int j = 0; j < 2; ++j) GRF_CUDA(cudaEventCreateWithFlags(&p->ev_part[j][i], cudaEventDisableTiming), "event");
    }
  }
  // each chunk's copy is split over several copy streams (several copy engines)
  const char* ncs_env = std::getenv("GRF_COPY_STREAMS");
  int ncs = ncs_env ? std::atoi(ncs_env) : 1;
  ncs = ncs < 1 ? 1 : (ncs > grf_plan_s::kCopyStreams ? grf_plan_s::kCopyStreams : ncs);
  int64_t idx = 0;
  for (int64_t f0 = 0; f0 < batch; f0 += per, ++idx) {
    const int64_t nb = batch - f0 < per ? batch - f0 : per;
    const int slot = (int)(idx & 1);
    if (idx >= 2) GRF_CUDA(cudaStreamWaitEvent(s, p->ev_copied[slot], 0), "wait copy");
    if (p->prec == GRF_FP64) {
      Plain64Geom g{};
      g.d = p->d;
      for (int i = 0; i < 3; ++i) g.n[i] = (int)p->n[i];
      for (int64_t b = 0; b < nb; ++b)
        LAUNCH(plain64_field(g, p->alg, seed + (uint64_t)(f0 + b), p->stab64, p->tw64, p->twax64, p->bufA, p->bufB,
                             (double*)p->stage[slot] + b * p->ntot, s),
               "FP64 plain field");
    } else if (p->mixed || p->kind == 2) {
      st = grf_sample(p, seed + (uint64_t)f0, nb, p->stage[slot], stream);
      if (st != GRF_OK) return st;
    } else {
      st = sample_chunk_fp32(p, seed, f0, nb, (float*)p->stage[slot], s);
      if (st != GRF_OK) return st;
    }
    GRF_CUDA(cudaEventRecord(p->ev_done[slot], s), "record");
    const size_t bytes = nb * field_bytes;
    const size_t part = ((bytes + ncs - 1) / ncs + 255) & ~size_t(255);
    for (int c = 0; c < ncs; ++c) {
      const size_t off = (size_t)c * part;
      if (off >= bytes) break;
      const size_t len = bytes - off < part ? bytes - off : part;
      GRF_CUDA(cudaStreamWaitEvent(p->copy_streams[c], p->ev_done[slot], 0), "wait compute");
      GRF_CUDA(cudaMemcpyAsync((char*)host_out + (size_t)f0 * field_bytes + off, (char*)p->stage[slot] + off, len,
                               cudaMemcpyDeviceToHost, p->copy_streams[c]),
               "copy to host");
      GRF_CUDA(cudaEventRecord(p->ev_part[slot][c], p->copy_streams[c]), "record");
      GRF_CUDA(cudaStreamWaitEvent(p->copy_stream, p->ev_part[slot][c], 0), "join copies");
    }
    GRF_CUDA(cudaEventRecord(p->ev_copied[slot], p->copy_stream), "record");
  }
  GRF_CUDA(cudaStreamSynchronize(p->copy_stream), "copy sync");
  return GRF_OK;
}

grf_status grf_backward(grf_plan p, uint64_t seed, int64_t batch, const void* grad_out, double* grad_params,
                        void* stream) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (p->kind != 0) return fail(GRF_ERR_INVALID_ARG, "the adjoint is built for periodic single-shape plans");
  if (!grad_out || !grad_params) return fail(GRF_ERR_INVALID_ARG, "NULL pointer");
  if (batch < 1 || batch > p->max_batch) return fail(GRF_ERR_INVALID_ARG, "batch must be in [1, max_batch]");
  if (p->prec != GRF_FP32 || p->alg != GRF_ALG_ONE_FFT || p->mixed)
    return fail(GRF_ERR_UNSUPPORTED, "the adjoint is built for FP32 Algorithm 2 plans on powers of two");
  if (!p->dstab) return fail(GRF_ERR_UNSUPPORTED, "the adjoint needs a Matern or Gaussian spectrum without normalize_discrete");
  if (p->d == 1 && p->M > 4096) return fail(GRF_ERR_UNSUPPORTED, "the adjoint is built for 1-D grids up to 8192");
  cudaStream_t s = (cudaStream_t)stream;
  const float* G = (const float*)grad_out;
  if (p->d == 1) {
    const HalfGeom g = half_geom(p, seed, 0);
    RowArgs r = row_args(p, g, batch, 1);
    r.inR = G;
    r.partial = grad_params;
    TLAUNCH(GRF_KERNEL_ROWS_1D, launch_row(ROW_LOAD_REAL, ROW_R2C_ADJ, p->row.P, r, row_grid(r), s), "1-D adjoint");
    return GRF_OK;
  }
  const int T = p->d == 2 ? p->T : 1;
  for (int64_t f0 = 0; f0 < batch; f0 += p->chunk) {
    const int64_t nb = batch - f0 < p->chunk ? batch - f0 : p->chunk;
    const HalfGeom g = half_geom(p, seed, f0);
    RowArgs r = row_args(p, g, nb, T);
    r.inR = G + f0 * p->ntot;
    r.outH = p->ws;
    TLAUNCH(GRF_KERNEL_ROWS_R2C, launch_row(ROW_LOAD_REAL, ROW_R2C, p->row.P, r, row_grid(r), s), "adjoint r2c");
    if (p->d == 3) {
      ColArgs b = col_axis2(p, g, p->ws, p->ws);
      TLAUNCH(GRF_KERNEL_COLUMNS, launch_col(COL_LOAD, COL_FWD, p->colB.P, b, col_grid(b, p->N1, nb), s), "adjoint axis 2");
    }
    ColArgs a = col_axis1(p, g, p->ws, nullptr, T);
    const dim3 grid = col_grid(a, 1, nb);
    const int64_t nblk = (int64_t)grid.x;
    st = ensure_partial(p, nblk * nb);
    if (st != GRF_OK) return st;
    a.partial = p->partial;
    TLAUNCH(GRF_KERNEL_COLUMNS, launch_col(COL_LOAD, COL_FWD_ADJ, p->colA.P, a, grid, s), "adjoint reduction");
    TLAUNCH(GRF_KERNEL_REDUCE, reduce_partials(p->partial, nblk, nb, grad_params + 3 * f0, s), "adjoint final sum");
  }
  return GRF_OK;
}

grf_status grf_rfft_forward(grf_plan p, int64_t batch, const void* in, void* out_halfspec, void* stream) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (p->kind != 0) return fail(GRF_ERR_INVALID_ARG, "rfft is built for periodic single-shape plans");
  if (!in || !out_halfspec) return fail(GRF_ERR_INVALID_ARG, "NULL pointer");
  if (batch < 1 || batch > p->max_batch) return fail(GRF_ERR_INVALID_ARG, "batch must be in [1, max_batch]");
  if (p->prec != GRF_FP32 || p->mixed) return fail(GRF_ERR_UNSUPPORTED, "rfft is built for FP32 plans on powers of two");
  if (p->d == 1 && p->M > 4096) return fail(GRF_ERR_UNSUPPORTED, "rfft is built for 1-D grids up to 8192");
  cudaStream_t s = (cudaStream_t)stream;
  const HalfGeom g = half_geom(p, 0, 0);
  float2* H = (float2*)out_halfspec;
  RowArgs r = row_args(p, g, batch, 1);
  r.inR = (const float*)in;
  r.outH = H;
  TLAUNCH(GRF_KERNEL_ROWS_R2C, launch_row(ROW_LOAD_REAL, ROW_R2C, p->row.P, r, row_grid(r), s), "rfft rows");
  if (p->d == 3) {
    ColArgs b = col_axis2(p, g, H, H);
    TLAUNCH(GRF_KERNEL_COLUMNS, launch_col(COL_LOAD, COL_FWD, p->colB.P, b, col_grid(b, p->N1, batch), s), "rfft axis 2");
  }
  if (p->d >= 2) {
    ColArgs a = col_axis1(p, g, H, H, 1);
    TLAUNCH(GRF_KERNEL_COLUMNS, launch_col(COL_LOAD, COL_FWD, p->colA.P, a, col_grid(a, 1, batch), s), "rfft axis 1");
  }
  return GRF_OK;
}

grf_status grf_batch_plan_create(grf_plan* out, int64_t count, const int* d, const int64_t* n, const double* L,
                                 const grf_spectrum* spec, int prec) {
  g_last_error.clear();
  if (!out) return fail(GRF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !d || !n || !L || !spec) return fail(GRF_ERR_INVALID_ARG, "bad batch description");
  if (prec != GRF_FP32) return fail(GRF_ERR_UNSUPPORTED, "batch plans are FP32");
  for (int64_t i = 0; i < count; ++i) {
    grf_status st = validate_spec(spec + i);
    if (st != GRF_OK) return st;
    if (spec[i].family > 1) return fail(GRF_ERR_UNSUPPORTED, "batch plans take Matern or Gaussian spectra");
  }
  grf_plan p = new (std::nothrow) grf_plan_s();
  if (!p) return fail(GRF_ERR_OOM, "host allocation");
  p->kind = 1;
  std::string err;
  grf_status st = batch_plan_build(&p->batch, count, d, n, L, spec, &err);
  if (st != GRF_OK) {
    free_plan(p);
    return fail(st, err);
  }
  cudaError_t e = dmalloc(&p->status, 1);
  if (e == cudaSuccess) e = cudaMemset(p->status, 0, sizeof(int));
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_fail(e, "status word");
  }
  *out = p;
  return GRF_OK;
}

grf_status grf_batch_sample(grf_plan p, uint64_t seed, void* const* out, void* stream) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (p->kind != 1) return fail(GRF_ERR_INVALID_ARG, "not a batch plan");
  if (!out) return fail(GRF_ERR_INVALID_ARG, "out is NULL");
  std::string err;
  st = batch_plan_sample(p->batch, seed, out, (cudaStream_t)stream, p->status, false, &err);
  return st == GRF_OK ? st : fail(st, err);
}

grf_status grf_batch_graph_launch(grf_plan p, uint64_t seed, void* const* out, void* stream) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (p->kind != 1) return fail(GRF_ERR_INVALID_ARG, "not a batch plan");
  if (!out) return fail(GRF_ERR_INVALID_ARG, "out is NULL");
  std::string err;
  st = batch_plan_sample(p->batch, seed, out, (cudaStream_t)stream, p->status, true, &err);
  return st == GRF_OK ? st : fail(st, err);
}

grf_status grf_batch_set_debug(grf_plan p, int withhold_field, double timeout_ms) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (p->kind != 1) return fail(GRF_ERR_INVALID_ARG, "not a batch plan");
  return batch_plan_debug(p->batch, withhold_field, timeout_ms);
}

grf_status grf_batch_set_mode(grf_plan p, int mode) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (p->kind != 1) return fail(GRF_ERR_INVALID_ARG, "not a batch plan");
  if (batch_plan_set_mode(p->batch, mode) != GRF_OK) return fail(GRF_ERR_INVALID_ARG, "batch mode must be 0 or 1");
  return GRF_OK;
}

grf_status grf_status_word(grf_plan p, void* stream) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  GRF_CUDA(cudaStreamSynchronize(s), "status sync");
  int h = 0;
  GRF_CUDA(cudaMemcpy(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
  GRF_CUDA(cudaMemset(p->status, 0, sizeof(int)), "status clear");
  return (grf_status)h;
}

grf_status grf_cov_origin(grf_plan p, uint64_t seed, int64_t count, double* sums, void* stream) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (p->kind == 1 || p->prec != GRF_FP32)
    return fail(GRF_ERR_UNSUPPORTED, "grf_cov_origin needs an FP32 single-shape plan");
  if (p->ntot > 0x7FFFFFFF) return fail(GRF_ERR_UNSUPPORTED, "grf_cov_origin: more than 2^31 - 1 points");
  if (count < 1) return fail(GRF_ERR_INVALID_ARG, "count must be >= 1");
  if (!sums) return fail(GRF_ERR_INVALID_ARG, "sums is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const int N = (int)p->ntot;  // points per field, flat C order
  const int64_t chunk = std::min<int64_t>(p->max_batch, (int64_t)65535 * 64);
  if (!p->cov_buf) {
    GRF_CUDA(dmalloc(&p->cov_buf, (size_t)(chunk * N)), "estimator field buffer");
    GRF_CUDA(dmalloc(&p->cov_partial, (size_t)(cov_origin_partial_count(chunk) * N)), "estimator partial sums");
  }
  for (int64_t f0 = 0; f0 < count; f0 += chunk) {
    const int64_t nb = std::min(chunk, count - f0);
    st = grf_sample(p, seed + (uint64_t)f0, nb, p->cov_buf, stream);
    if (st != GRF_OK) return st;
    LAUNCH(launch_cov_origin(p->cov_buf, nb, N, p->cov_partial, sums, s), "covariance estimator");
  }
  return GRF_OK;
}

grf_status grf_philox_words(uint64_t key, uint32_t tag, uint64_t q0, int64_t count, uint32_t* out_words,
                            void* stream) {
  if (!out_words || count < 0) return fail(GRF_ERR_INVALID_ARG, "bad philox_words arguments");
  if (count == 0) return GRF_OK;
  LAUNCH(philox_words(key, tag, q0, count, out_words, (cudaStream_t)stream), "philox words");
  return GRF_OK;
}

grf_status grf_plan_timing(grf_plan p, int64_t cap) {
  grf_status st = check_plan(p);
  if (st != GRF_OK) return st;
  if (cap < 0) return fail(GRF_ERR_INVALID_ARG, "cap must be >= 0");
  for (cudaEvent_t e : p->tev) cudaEventDestroy(e);
  p->tev.clear();
  p->tkind.assign((size_t)cap, -1);
  p->tev.resize((size_t)(2 * cap), nullptr);
  for (auto& e : p->tev) GRF_CUDA(cudaEventCreate(&e), "timing event");
  p->tcap = cap;
  p->tused = 0;
  return GRF_OK;
}

int64_t grf_plan_timing_read(grf_plan p, int* kinds, float* ms, int64_t cap_out) {
  if (!p) return -1;
  const int64_t n = p->tused;
  const int64_t rec = n < p->tcap ? n : p->tcap;
  for (int64_t i = 0; i < rec && i < cap_out; ++i) {
    float t = 0.f;
    if (cudaEventSynchronize(p->tev[2 * i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, p->tev[2 * i], p->tev[2 * i + 1]) != cudaSuccess)
      t = -1.f;
    if (kinds) kinds[i] = p->tkind[i];
    if (ms) ms[i] = t;
  }
  p->tused = 0;
  return n;
}

int64_t grf_plan_query(grf_plan p, int key) {
  if (!p) return -1;
  if (p->kind == 1) {
    if (key == 0) return batch_plan_total_points(p->batch);
    return -1;
  }
  if (p->kind == 2) {
    switch (key) {
      case 0: return p->ntot;
      case 3: return p->d;
      case 4: return p->n[0];
      case 5: return p->n[1];
      case 6: return p->n[2];
      case 16: return p->bc;
      default: return -1;
    }
  }
  switch (key) {
    case 0: return p->ntot;
    case 1: return p->hsize;
    case 2: return (int64_t)(p->chunk * p->hsize * (int64_t)sizeof(float2));
    case 3: return p->d;
    case 4: return p->n[0];
    case 5: return p->n[1];
    case 6: return p->n[2];
    case 7: return p->T;
    case 8: return p->colA.P;
    case 9: return p->colA.C;
    case 10: return p->row.P;
    case 11: return p->row.C;
    case 12: return p->pipe;
    case 13: return p->colB.P;
    case 14: return p->colB.C;
    case 15: return p->row_tma;
    case 17: return p->plane_R;
    default: return -1;
  }
}

grf_status grf_plan_destroy(grf_plan p) {
  if (!p) return GRF_OK;
  cudaSetDevice(p->device);
  free_plan(p);
  return GRF_OK;
}

}  // extern "C"
