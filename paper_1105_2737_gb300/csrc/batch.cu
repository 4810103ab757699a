// Uneven batches: thousands of fields of different shapes, dimensions and
// Matern / Gaussian parameters sampled (Algorithm 2, FP32) by ONE persistent
// kernel launch, optionally replayed from a CUDA graph.
//
// Work decomposition.  Every field is a short chain of passes (2-D: noise +
// axis-1 columns, then c2r rows; 3-D: noise + axis-1 columns, axis-2 columns,
// c2r rows; 1-D: the two stages of the four-step c2r).  A pass is split into
// tiles (a few columns or rows, one CTA-sized piece of work).  The queue holds
// every (pass, tile) of every field, all first passes first, then all second
// passes, then all third passes.  Persistent CTAs pop tiles in queue order
// with one atomic; a tile of pass p of field f first waits until the per-field
// counter of pass p - 1 reaches that pass's tile count.  Because tiles are
// popped in queue order, everything a tile waits for has already been popped
// by a running CTA, so the waits end.  Each wait is still bounded (iteration
// cap and a %globaltimer deadline): on expiry the kernel records
// GRF_ERR_TIMEOUT in the plan's status word, raises an abort flag that makes
// every CTA stop taking tiles, and returns.
//
// Schedules: threads per tile and CTAs per SM are chosen by a tuner that
// times the candidates on the first call and keeps the winner in a cache file
// (GRF_TUNE_CACHE, default $HOME/.cache/grf_gb300_tune.txt) keyed by the GPU
// name and the batch's shape signature.
#include "batch.h"
#include "bodies.cuh"
#include "tune_cache.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <sstream>
#include <tuple>
#include <string>
#include <vector>

namespace grf {

enum JobKind { JOB_COL_NOISE = 0, JOB_COL_LOAD = 1, JOB_ROW_C2R = 2, JOB_FS1 = 3, JOB_FS2 = 4 };

struct Job {
  int kind, pass, nthr;
  int gx;         // tile -> (bx = tile % gx, by = tile / gx)
  int field;      // index in the batch (seed + field is its Philox key)
  int need_prev;  // tiles of the previous pass of this field
  ColArgs col;
  RowArgs row;
  FourStepArgs fs;
};

struct BatchParams {
  const Job* jobs;
  const int2* items;  // (job, tile), in queue order
  int nitems;
  int* queue;
  int* counters;  // 3 per field
  int* abort_flag;
  int* status;
  float* const* outs;
  uint64_t seed;
  long long timeout_ns;
  int withhold_field;  // test hook: this field's first pass never reports done (-1: off)
};

constexpr int kBatchThreads = 256;
constexpr long long kDefaultTimeoutNs = 2000000000LL;  // 2 s
constexpr unsigned kSpinCap = 1u << 26;

GRF_DEV unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

GRF_DEV int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait for counter >= need.  Returns 1 when it is, 0 on abort or timeout.
GRF_DEV int wait_counter(const int* ctr, int need, const BatchParams& b) {
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned it = 0;; ++it) {
    if (ld_acquire(ctr) >= need) return 1;
    if (ld_acquire(b.abort_flag)) return 0;
    if (it > kSpinCap || (long long)(globaltimer_ns() - t0) > b.timeout_ns) {
      atomicExch(b.status, (int)GRF_ERR_TIMEOUT);
      atomicExch(b.abort_flag, 1);
      return 0;
    }
    __nanosleep(256);
  }
}

// One call per job kind, kept out of line so that each body gets its own
// register allocation instead of the union of all five.
__device__ __noinline__ void run_col_noise(const ColArgs& a, int bx, int by, int nthr, float2* sm) {
  col_body<16, COL_NOISE, COL_INV>(a, bx, by, 0, 0, nthr, sm);
}
__device__ __noinline__ void run_col_noise_pair(const ColArgs& a, int bx, int by, int nthr, float2* sm) {
  col_body_pair<16, COL_NOISE, COL_INV>(a, CtaCoordsVal{bx, by, 0}, nthr, sm);
}
__device__ __noinline__ void run_col_load_pair(const ColArgs& a, int bx, int by, int nthr, float2* sm) {
  col_body_pair<16, COL_LOAD, COL_INV>(a, CtaCoordsVal{bx, by, 0}, nthr, sm);
}
__device__ __noinline__ void run_row_c2r(const RowArgs& a, int bx, int nthr, float2* sm) {
  row_body<16, ROW_LOAD_Z, ROW_C2R>(a, bx, nthr, sm);
}
__device__ __noinline__ void run_fs1(const FourStepArgs& a, int bx, int nthr, float2* sm) {
  fourstep1_body<16>(a, bx, 0, nthr, sm);
}
__device__ __noinline__ void run_fs2(const FourStepArgs& a, int bx, int nthr, float2* sm) {
  fourstep2_body<16>(a, bx, 0, nthr, sm);
}

__global__ void __launch_bounds__(kBatchThreads, 2) batch_kernel(BatchParams b) {
  extern __shared__ float2 sm[];
  __shared__ Job s_job;
  __shared__ int s_item, s_ok;
  const int t = threadIdx.x;
  for (;;) {
    if (t == 0) {
      const int i = atomicAdd(b.queue, 1);
      s_item = (i < b.nitems && !ld_acquire(b.abort_flag)) ? i : -1;
    }
    __syncthreads();
    const int i = s_item;
    if (i < 0) break;
    const int2 it = b.items[i];
    {  // stage the job descriptor in shared memory
      const int* src = reinterpret_cast<const int*>(b.jobs + it.x);
      int* dst = reinterpret_cast<int*>(&s_job);
      for (int w = t; w < (int)(sizeof(Job) / sizeof(int)); w += kBatchThreads) dst[w] = src[w];
    }
    __syncthreads();
    if (t == 0) {
      s_job.col.g.seed = b.seed;
      s_job.row.g.seed = b.seed;
      s_job.fs.seed = b.seed;
      if (s_job.kind == JOB_ROW_C2R) s_job.row.outR = b.outs[s_job.field];
      if (s_job.kind == JOB_FS2) s_job.fs.out = b.outs[s_job.field];
      s_ok = s_job.pass == 0 ? 1 : wait_counter(b.counters + 3 * s_job.field + s_job.pass - 1, s_job.need_prev, b);
    }
    __syncthreads();
    if (!s_ok) break;
    const int bx = it.y % s_job.gx, by = it.y / s_job.gx;
    const int nthr = s_job.nthr;
    if (t < nthr) {
      switch (s_job.kind) {
        case JOB_COL_NOISE:
          if (s_job.col.zpair) run_col_noise_pair(s_job.col, bx, by, nthr, sm);
          else run_col_noise(s_job.col, bx, by, nthr, sm);
          break;
        case JOB_COL_LOAD: run_col_load_pair(s_job.col, bx, by, nthr, sm); break;
        case JOB_ROW_C2R: run_row_c2r(s_job.row, bx, nthr, sm); break;
        case JOB_FS1: run_fs1(s_job.fs, bx, nthr, sm); break;
        default: run_fs2(s_job.fs, bx, nthr, sm); break;
      }
    }
    __syncthreads();
    if (t == 0 && !(s_job.pass == 0 && s_job.field == b.withhold_field)) {
      __threadfence();  // the tile's writes (ordered by the barrier) before the count
      atomicAdd(b.counters + 3 * s_job.field + s_job.pass, 1);
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct FieldInfo {
  int d;
  int n[3];
  double L[3];
  grf_spectrum spec;
  int64_t points, stab_off, ws_off;
};

struct BatchPlan {
  int64_t count = 0;
  int64_t total_points = 0;
  std::vector<FieldInfo> fields;
  int twmax = 0;
  float2* tw = nullptr;
  float* stabs = nullptr;
  float2* ws = nullptr;
  Job* jobs = nullptr;
  int2* items = nullptr;
  int njobs = 0, nitems = 0;
  int* counters = nullptr;  // 3 per field, then queue, abort flag
  float** outs = nullptr;
  size_t smem = 0;
  int num_sms = 0;
  // schedule
  int tile_threads = 256;
  int ctas_per_sm = 2;
  bool tuned = false;
  std::string signature;
  // graph replay
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphNode_t knode = nullptr;
  std::vector<void*> graph_outs;
  std::vector<void*> cur_outs;
  BatchParams kparams{};
  int withhold = -1;
  long long timeout_ns = kDefaultTimeoutNs;
  // Per-shape launches (the default mode): fields grouped by shape, each class
  // sampled by the plan kernels with one launch index z per field, the classes
  // spread over several streams; one captured graph replays them all.
  struct ShapeClass {
    int d = 1, n[3] = {1, 1, 1};
    int64_t nf = 0, first = 0;      // fields, offset in the class-ordered arrays
    int64_t stab_off = 0, fold = 0; // tables: base and stride
    int64_t ws_off = 0, wstride = 0;
    int64_t points = 0;
    int stream = 0;
    int64_t stabT_off = -1;  // 1-D four-step: s_k along k2, M per field
  };
  float* stabsT = nullptr;
  int mode = 0;  // 0: per-shape launches, 1: one persistent kernel
  std::vector<ShapeClass> classes;
  std::vector<int64_t> class_order;  // batch index of each class-ordered slot
  int64_t* zfield = nullptr;         // device copy of class_order
  float** zouts = nullptr;           // output pointers, class-ordered
  uint64_t* seed_dev = nullptr;
  int* status_dev = nullptr;  // the plan's status word (the plane path's bulk-copy waits report here)
  static constexpr int kStreams = 8;
  cudaStream_t cstreams[kStreams] = {};
  cudaEvent_t cfork = nullptr, cjoin[kStreams] = {};
  cudaGraphExec_t cexec = nullptr;
  cudaGraph_t cgraph = nullptr;
  std::vector<void*> cgraph_outs;
};

namespace {

bool pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
int lg2(int64_t x) {
  int r = 0;
  while ((int64_t(1) << r) < x) ++r;
  return r;
}
int64_t npow2(int64_t x) {
  int64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Columns (or rows) per tile for transforms of length len: `target` threads of
// 16 points, at least one warp, no more than the columns there are.
int tile_cols(int len, int64_t ncols, int target) {
  const int tpt = len / 16;
  int C = target / tpt;
  if (C < 1) C = 1;
  const int cmin = 32 / tpt > 1 ? 32 / tpt : 1;
  const int64_t cp = npow2(ncols);
  if (C > cp) C = (int)cp;
  if (C < cmin) C = cmin;
  return C;
}

cudaError_t build_jobs(BatchPlan* b) {
  std::vector<Job> jobs;
  std::vector<int2> items[3];
  const float2* tws = b->tw + 2 * b->twmax;
  for (int64_t i = 0; i < b->count; ++i) {
    const FieldInfo& f = b->fields[i];
    const int d = f.d;
    const int Nd = f.n[d - 1], M = Nd / 2;
    HalfGeom g{};
    g.d = d;
    g.N1 = d >= 2 ? f.n[0] : 1;
    g.Nmid = d == 3 ? f.n[1] : 1;
    g.M = M;
    g.Q = (uint32_t)(M / 2 + 1);
    g.seed = 0;
    g.field0 = i;  // key = seed + i
    g.stab = b->stabs + f.stab_off;
    g.trig = b->tw + 256;
    float2* ws = b->ws + f.ws_off;
    auto add = [&](Job j, int tiles) {
      const int id = (int)jobs.size();
      jobs.push_back(j);
      for (int t = 0; t < tiles; ++t) items[j.pass].push_back(make_int2(id, t));
      return tiles;
    };
    if (d == 1) {
      const int lm = lg2(M);
      FourStepArgs fs{};
      fs.B = 1 << ((lm + 1) / 2);
      fs.A = M / fs.B;
      fs.logA = lg2(fs.A);
      fs.logB = lg2(fs.B);
      fs.M = M;
      fs.N = Nd;
      const int C1 = std::min(tile_cols(fs.B, fs.A, b->tile_threads), fs.A);
      const int C2 = std::min(tile_cols(fs.A, fs.B, b->tile_threads), fs.B);
      fs.T = C1;
      fs.logT = lg2(C1);
      fs.Y = ws;
      fs.Yin = ws;
      fs.twA = b->tw + fs.A;
      fs.twB = b->tw + fs.B;
      fs.twM = b->tw + M;
      fs.twN = b->tw + Nd;
      fs.tws = tws;
      fs.stab = g.stab;
      fs.trig = g.trig;
      fs.field0 = i;
      Job j1{};
      j1.kind = JOB_FS1;
      j1.pass = 0;
      j1.field = (int)i;
      j1.fs = fs;
      j1.fs.C = C1;
      j1.nthr = C1 * fs.B / 16;
      j1.gx = fs.A / C1;
      const int t1 = add(j1, j1.gx);
      Job j2 = j1;
      j2.kind = JOB_FS2;
      j2.pass = 1;
      j2.fs.C = C2;
      j2.nthr = C2 * fs.A / 16;
      j2.gx = fs.B / C2;
      j2.need_prev = t1;
      add(j2, j2.gx);
      continue;
    }
    // 2-D and 3-D: axis-1 columns with the noise
    ColArgs a{};
    a.N = g.N1;
    a.logN = lg2(g.N1);
    a.ncols = (int64_t)g.Nmid * (M + 1);
    a.C = tile_cols(a.N, a.ncols, b->tile_threads);
    a.T = 1;
    a.logT = 0;
    a.out = ws;
    a.tw = b->tw + g.N1;
    a.tws = tws;
    a.g = g;
    int64_t slots = a.ncols;
    if (d == 2) {  // the last column pass writes Z of the c2r split
      a.zpair = 1;
      a.twz = b->tw + Nd;
      slots = M / 2 + 1;
      a.C = tile_cols(a.N, slots, b->tile_threads);
    }
    Job ja{};
    ja.kind = JOB_COL_NOISE;
    ja.pass = 0;
    ja.field = (int)i;
    ja.col = a;
    ja.nthr = a.C * a.N / 16;
    ja.gx = (int)((slots + a.C - 1) / a.C);
    int prev = add(ja, ja.gx);
    int pass = 1;
    if (d == 3) {
      ColArgs a2{};
      a2.N = g.Nmid;
      a2.logN = lg2(g.Nmid);
      a2.ncols = M + 1;
      a2.zpair = 1;  // the last column pass writes Z of the c2r split
      a2.twz = b->tw + Nd;
      a2.C = tile_cols(a2.N, M / 2 + 1, b->tile_threads);
      a2.T = 1;
      a2.logT = 0;
      a2.ostride = (int64_t)g.Nmid * (M + 1);
      a2.in = ws;
      a2.out = ws;
      a2.tw = b->tw + g.Nmid;
      a2.tws = tws;
      a2.g = g;
      Job jb{};
      jb.kind = JOB_COL_LOAD;
      jb.pass = 1;
      jb.field = (int)i;
      jb.col = a2;
      jb.nthr = a2.C * a2.N / 16;
      jb.gx = (int)((M / 2 + 1 + a2.C - 1) / a2.C);
      jb.need_prev = prev;
      prev = add(jb, jb.gx * g.N1);
      pass = 2;
    }
    RowArgs r{};
    r.M = M;
    r.logM = lg2(M);
    r.rows_per_field = (int64_t)g.N1 * g.Nmid;
    r.nrows = r.rows_per_field;
    r.C = tile_cols(M, r.nrows, b->tile_threads);
    r.T = 1;
    r.logT = 0;
    r.inH = ws;
    r.twM = b->tw + M;
    r.twN = b->tw + Nd;
    r.tws = tws;
    r.g = g;
    Job jr{};
    jr.kind = JOB_ROW_C2R;
    jr.pass = pass;
    jr.field = (int)i;
    jr.row = r;
    jr.nthr = r.C * M / 16;
    jr.gx = (int)(r.nrows / r.C);
    jr.need_prev = prev;
    add(jr, jr.gx);
  }
  std::vector<int2> all;
  // Within a pass, tiles of one body (job kind) run together, so the CTAs on
  // an SM share their instructions; waits only reach back to earlier passes,
  // so the order inside a pass keeps every wait finite.
  auto kind_rank = [&](const int2& it) {
    const Job& j = jobs[it.x];
    return j.kind * 2 + (j.kind == JOB_COL_NOISE && j.col.zpair ? 1 : 0);
  };
  for (int p = 0; p < 3; ++p) {
    std::stable_sort(items[p].begin(), items[p].end(),
                     [&](const int2& x, const int2& y) { return kind_rank(x) < kind_rank(y); });
    all.insert(all.end(), items[p].begin(), items[p].end());
  }
  cudaFree(b->jobs);
  cudaFree(b->items);
  b->jobs = nullptr;
  b->items = nullptr;
  cudaError_t e = cudaMalloc(&b->jobs, jobs.size() * sizeof(Job));
  if (e == cudaSuccess) e = cudaMalloc(&b->items, all.size() * sizeof(int2));
  if (e == cudaSuccess) e = cudaMemcpy(b->jobs, jobs.data(), jobs.size() * sizeof(Job), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->items, all.data(), all.size() * sizeof(int2), cudaMemcpyHostToDevice);
  b->njobs = (int)jobs.size();
  b->nitems = (int)all.size();
  size_t smem = 3 * 32 * sizeof(double);
  for (const Job& j : jobs) {
    size_t need = 0;
    if (j.kind == JOB_COL_NOISE || j.kind == JOB_COL_LOAD)
      need = j.col.zpair ? col_pair_smem_bytes(j.col.N, j.col.C) : col_smem_bytes(j.col.N, j.col.C);
    else if (j.kind == JOB_ROW_C2R) need = row_smem_bytes(j.row.M, j.row.C);
    else need = col_smem_bytes(j.kind == JOB_FS1 ? j.fs.B : j.fs.A, j.fs.C);
    smem = std::max(smem, need);
  }
  b->smem = smem;
  return e;
}

}  // namespace
}  // namespace grf

namespace grf {
namespace {

cudaError_t launch_batch(BatchPlan* b, uint64_t seed, cudaStream_t s, int* status) {
  cudaError_t e = cudaMemsetAsync(b->counters, 0, (size_t)(3 * b->count + 2) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  BatchParams p{};
  p.jobs = b->jobs;
  p.items = b->items;
  p.nitems = b->nitems;
  p.counters = b->counters;
  p.queue = b->counters + 3 * b->count;
  p.abort_flag = b->counters + 3 * b->count + 1;
  p.status = status;
  p.outs = b->outs;
  p.seed = seed;
  p.timeout_ns = b->timeout_ns;
  p.withhold_field = b->withhold;
  e = prepare_kernel((const void*)batch_kernel, kBatchThreads, b->smem);
  if (e != cudaSuccess) return e;
  const int grid = b->num_sms * b->ctas_per_sm;
  batch_kernel<<<grid, kBatchThreads, b->smem, s>>>(p);
  b->kparams = p;
  return cudaGetLastError();
}

cudaError_t set_outs(BatchPlan* b, void* const* out, cudaStream_t s) {
  std::vector<void*> v(out, out + b->count);
  if (v == b->cur_outs) return cudaSuccess;
  // pageable source: the copy is staged before the call returns, ordered on s
  cudaError_t e = cudaMemcpyAsync(b->outs, v.data(), v.size() * sizeof(void*), cudaMemcpyHostToDevice, s);
  std::vector<void*> z(b->count);
  for (int64_t k = 0; k < b->count; ++k) z[k] = v[b->class_order[k]];
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->zouts, z.data(), z.size() * sizeof(void*), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) b->cur_outs = v;
  return e;
}

// One shape class: the plan kernels over its nf fields (launch index z =
// the class-ordered slot first + z), on stream s.
cudaError_t launch_class(BatchPlan* b, const BatchPlan::ShapeClass& c, cudaStream_t s) {
  const int d = c.d;
  const int Nd = c.n[d - 1], M = Nd / 2;
  const int N1 = d >= 2 ? c.n[0] : 1, Nmid = d == 3 ? c.n[1] : 1;
  const float2* tws = b->tw + 2 * b->twmax;
  HalfGeom g{};
  g.d = d;
  g.N1 = N1;
  g.Nmid = Nmid;
  g.M = M;
  g.Q = (uint32_t)(M / 2 + 1);
  g.stab = b->stabs + c.stab_off;
  g.stab_zstride = c.fold;
  g.zfield = b->zfield + c.first;
  g.seed_ptr = b->seed_dev;
  g.trig = b->tw + 256;
  float2* ws = b->ws + c.ws_off;
  float* const* zout = b->zouts + c.first;
  const int64_t nf = c.nf;
  cudaError_t e;
  if (d == 1 && M <= 4096) {
    RowArgs r{};
    r.M = M;
    r.logM = lg2(M);
    r.C = tile_cols(M, nf, 256);
    r.rows_per_field = 1;
    r.nrows = nf;
    r.T = 1;
    r.twM = b->tw + M;
    r.twN = b->tw + Nd;
    r.tws = tws;
    r.g = g;
    r.zout = zout;
    return launch_row(ROW_NOISE_H, ROW_C2R, 16, r, dim3((unsigned)((nf + r.C - 1) / r.C)), s);
  }
  if (d == 1) {
    const int lm = lg2(M);
    FourStepArgs fs{};
    fs.B = 1 << ((lm + 1) / 2);
    fs.A = M / fs.B;
    fs.logA = lg2(fs.A);
    fs.logB = lg2(fs.B);
    fs.M = M;
    fs.N = Nd;
    const int C1 = std::min(4096 / fs.B, fs.A), C2 = std::min(4096 / fs.A, fs.B);
    fs.T = C1 / 2;  // stage 1 in mirror pairs: C1 / 2 pairs per CTA
    fs.logT = lg2(C1 / 2);
    fs.Y = ws;
    fs.Yin = ws;
    fs.twA = b->tw + fs.A;
    fs.twB = b->tw + fs.B;
    fs.twM = b->tw + M;
    fs.twN = b->tw + Nd;
    fs.tws = tws;
    fs.stab = g.stab;
    fs.stab_zstride = c.fold;
    fs.stabT = b->stabsT + c.stabT_off;
    fs.stabT_zstride = M;
    fs.tw2B = b->tw + 2 * fs.B;
    fs.twMA = b->tw + fs.A;
    fs.trig = g.trig;
    fs.zfield = g.zfield;
    fs.seed_ptr = g.seed_ptr;
    fs.zout = zout;
    fs.C = C1;
    if ((e = launch_fourstep(3, 16, fs, nf, s)) != cudaSuccess) return e;
    fs.C = C2;
    return launch_fourstep(2, 16, fs, nf, s);
  }
  if (d == 3 && plane3_radix(N1, Nmid, M)) {  // two passes: whole (sub-)planes in shared memory
    PlaneArgs pl{};
    pl.N1 = N1;
    pl.N2 = Nmid;
    pl.M = M;
    pl.R = plane3_radix(N1, Nmid, M);
    pl.Q = Nmid / pl.R;
    pl.S3 = M + 2;
    pl.ws = ws;
    pl.tw = b->tw;
    pl.tws = tws;
    pl.status = b->status_dev;
    pl.zout = zout;
    ColArgs a{};
    a.N = N1;
    a.logN = lg2(N1);
    a.ncols = (int64_t)Nmid * (M + 1);
    a.T = 1;
    a.logT = 0;
    a.bstride = (int64_t)N1 * Nmid * pl.S3;
    a.out = ws;
    a.tw = b->tw + N1;
    a.tws = tws;
    a.plane_is_k1 = 1;
    a.g = g;
    if (N1 >= 256) {
      e = launch_plane3_noise(a, pl, nf, s);
    } else {
      a.pitch3 = pl.S3;
      a.C = tile_cols(N1, a.ncols, 256);
      e = launch_col(COL_NOISE, COL_INV, 16, a, dim3((unsigned)((a.ncols + a.C - 1) / a.C), 1, (unsigned)nf), s);
    }
    if (e != cudaSuccess) return e;
    return launch_plane3_c2r(pl, nf, s);
  }
  const int T = (d == 2 && N1 >= 256) ? 8 : 1;
  const int64_t hsize = (int64_t)N1 * Nmid * (M + 1);
  ColArgs a{};
  a.N = N1;
  a.logN = lg2(N1);
  a.ncols = (int64_t)Nmid * (M + 1);
  a.T = T;
  a.logT = lg2(T);
  a.bstride = hsize;
  a.out = ws;
  a.tw = b->tw + N1;
  a.tws = tws;
  a.plane_is_k1 = 1;
  a.g = g;
  int64_t slots = a.ncols;
  if (d == 2) {
    a.zpair = 1;
    a.twz = b->tw + Nd;
    slots = M / 2 + 1;
  }
  a.C = tile_cols(N1, slots, 256);
  e = launch_col(COL_NOISE, COL_INV, 16, a, dim3((unsigned)((slots + a.C - 1) / a.C), 1, (unsigned)nf), s);
  if (e != cudaSuccess) return e;
  if (d == 3) {
    ColArgs a2{};
    a2.N = Nmid;
    a2.logN = lg2(Nmid);
    a2.ncols = M + 1;
    a2.zpair = 1;
    a2.twz = b->tw + Nd;
    a2.C = tile_cols(Nmid, M / 2 + 1, 256);
    a2.T = 1;
    a2.logT = 0;
    a2.ostride = (int64_t)Nmid * (M + 1);
    a2.bstride = hsize;
    a2.in = ws;
    a2.out = ws;
    a2.tw = b->tw + Nmid;
    a2.tws = tws;
    a2.g = g;
    e = launch_col(COL_LOAD, COL_INV, 16, a2, dim3((unsigned)((M / 2 + 1 + a2.C - 1) / a2.C), (unsigned)N1, (unsigned)nf), s);
    if (e != cudaSuccess) return e;
  }
  RowArgs r{};
  r.M = M;
  r.logM = lg2(M);
  r.rows_per_field = (int64_t)N1 * Nmid;
  r.nrows = nf * r.rows_per_field;
  r.C = tile_cols(M, r.nrows, 256);
  r.T = T;
  r.logT = lg2(T);
  r.inH = ws;
  r.twM = b->tw + M;
  r.twN = b->tw + Nd;
  r.tws = tws;
  r.g = g;
  r.zout = zout;
  return launch_row(ROW_LOAD_Z, ROW_C2R, 16, r, dim3((unsigned)((r.nrows + r.C - 1) / r.C)), s);
}

// All classes: forked from s onto the class streams and joined back into s.
cudaError_t launch_classes(BatchPlan* b, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(b->cfork, s);
  for (int q = 0; q < BatchPlan::kStreams && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(b->cstreams[q], b->cfork, 0);
  for (const auto& c : b->classes) {
    if (e != cudaSuccess) break;
    e = launch_class(b, c, b->cstreams[c.stream]);
  }
  for (int q = 0; q < BatchPlan::kStreams && e == cudaSuccess; ++q) {
    e = cudaEventRecord(b->cjoin[q], b->cstreams[q]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->cjoin[q], 0);
  }
  return e;
}

// Time the current schedule: the fastest of three launches after a warm-up
// launch (one launch of a small batch is too short to time alone).
float time_launch(BatchPlan* b, uint64_t seed, cudaStream_t s, int* status) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch_batch(b, seed, s, status);
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, s);
    launch_batch(b, seed, s, status);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 1e30f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = 1e30f;
    best = ms < best ? ms : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// The tuner: threads per tile x CTAs per SM, timed on the caller's outputs.
cudaError_t tune(BatchPlan* b, uint64_t seed, cudaStream_t s, int* status) {
  float best = 1e30f;
  int bt = b->tile_threads, bc = b->ctas_per_sm;
  for (int tt : {128, 256}) {
    b->tile_threads = tt;
    cudaError_t e = build_jobs(b);
    if (e != cudaSuccess) return e;
    // CTAs per SM that fit this schedule's shared memory (the dynamic
    // shared-memory limit is raised before the occupancy query)
    e = prepare_kernel((const void*)batch_kernel, kBatchThreads, b->smem);
    if (e != cudaSuccess) return e;
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel, kBatchThreads, b->smem);
    if (occ < 1) occ = 1;
    for (int cps = 1; cps <= std::min(occ, 4); ++cps) {
      b->ctas_per_sm = cps;
      const float ms = time_launch(b, seed, s, status);
      if (ms < best) {
        best = ms;
        bt = tt;
        bc = cps;
      }
    }
  }
  b->tile_threads = bt;
  b->ctas_per_sm = bc;
  cudaError_t e = build_jobs(b);
  if (e != cudaSuccess) return e;
  b->tuned = true;
  tune_cache_store(b->signature, {bt, bc});
  return cudaSuccess;
}

void drop_graph(BatchPlan* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->knode = nullptr;
  b->graph_outs.clear();
}

}  // namespace

grf_status batch_plan_build(BatchPlan** out, int64_t count, const int* d, const int64_t* n, const double* L,
                            const grf_spectrum* spec, std::string* err) {
  *out = nullptr;
  if (count > (1 << 24)) {
    *err = "too many fields";
    return GRF_ERR_INVALID_ARG;
  }
  BatchPlan* b = new BatchPlan();
  b->count = count;
  b->fields.resize(count);
  int64_t stab_total = 0, ws_total = 0;
  int twmax = 256;  // the length-256 table also serves Box-Muller's coarse angles
  std::ostringstream sig;
  sig << "batch|" << tune_gpu_name() << "|" << count;
  uint64_t hsh = 1469598103934665603ull;
  for (int64_t i = 0; i < count; ++i) {
    FieldInfo& f = b->fields[i];
    f.d = d[i];
    if (f.d < 1 || f.d > 3) {
      delete b;
      *err = "field dimension must be 1, 2 or 3";
      return GRF_ERR_INVALID_ARG;
    }
    f.points = 1;
    for (int k = 0; k < 3; ++k) {
      f.n[k] = k < f.d ? (int)n[3 * i + k] : 1;
      f.L[k] = k < f.d ? L[3 * i + k] : 1.0;
      if (k < f.d) {
        if (n[3 * i + k] < 2 || (n[3 * i + k] & 1) || !(f.L[k] > 0)) {
          delete b;
          *err = "every N_i must be even and every L_i > 0";
          return GRF_ERR_INVALID_ARG;
        }
        const bool ok = pow2(f.n[k]) && (f.d == 1 ? (f.n[k] >= 1024 && f.n[k] <= (1 << 22))
                                                   : (f.n[k] >= 32 && f.n[k] <= 4096));
        if (!ok) {
          delete b;
          *err = "batch plans take powers of two: 1-D 1024..2^22, 2-D/3-D sides 32..4096";
          return GRF_ERR_UNSUPPORTED;
        }
        f.points *= f.n[k];
        twmax = std::max(twmax, f.n[k]);
        hsh = (hsh ^ (uint64_t)f.n[k]) * 1099511628211ull;
      }
    }
    hsh = (hsh ^ (uint64_t)(f.d + 7)) * 1099511628211ull;
    f.spec = spec[i];
    b->total_points += f.points;
  }
  // shape classes; a class's tables and workspaces are contiguous with a
  // fixed stride, so that one launch can index them by z
  {
    std::vector<int64_t> idx(count);
    for (int64_t i = 0; i < count; ++i) idx[i] = i;
    auto key = [&](int64_t i) {
      const FieldInfo& f = b->fields[i];
      return std::make_tuple(f.d, f.n[0], f.n[1], f.n[2]);
    };
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return key(x) < key(y); });
    for (int64_t k = 0; k < count;) {
      int64_t e = k;
      while (e < count && key(idx[e]) == key(idx[k])) ++e;
      BatchPlan::ShapeClass c;
      const FieldInfo& f0 = b->fields[idx[k]];
      c.d = f0.d;
      for (int q = 0; q < 3; ++q) c.n[q] = f0.n[q];
      c.nf = e - k;
      const int M = f0.n[f0.d - 1] / 2;
      const int N1 = f0.d >= 2 ? f0.n[0] : 1, Nmid = f0.d == 3 ? f0.n[1] : 1;
      c.fold = (int64_t)(N1 / 2 + 1) * (Nmid / 2 + 1) * (M + 1);
      c.wstride = f0.d == 1 ? M : (int64_t)N1 * Nmid * (M + 1);
      if (f0.d == 3 && plane3_radix(N1, Nmid, M)) c.wstride = (int64_t)plane3_ws_entries(N1, Nmid, M);
      c.stab_off = stab_total;
      c.ws_off = ws_total;
      c.points = f0.points * c.nf;
      for (int64_t r = k; r < e; ++r) {
        FieldInfo& f = b->fields[idx[r]];
        f.stab_off = stab_total + (r - k) * c.fold;
        f.ws_off = ws_total + (r - k) * c.wstride;
      }
      stab_total = (stab_total + c.nf * c.fold + 63) & ~int64_t(63);
      ws_total = (ws_total + c.nf * c.wstride + 31) & ~int64_t(31);
      b->classes.push_back(c);
      k = e;
    }
    // the largest classes first, each on the stream with the least work so far
    std::stable_sort(b->classes.begin(), b->classes.end(),
                     [](const BatchPlan::ShapeClass& x, const BatchPlan::ShapeClass& y) { return x.points > y.points; });
    int64_t load[BatchPlan::kStreams] = {};
    for (auto& c : b->classes) {
      int best = 0;
      for (int q = 1; q < BatchPlan::kStreams; ++q)
        if (load[q] < load[best]) best = q;
      c.stream = best;
      load[best] += c.points;
      c.first = (int64_t)b->class_order.size();
      // fields of the class in batch order: their offsets are increasing
      std::vector<int64_t> mem;
      for (int64_t i = 0; i < count; ++i) {
        const FieldInfo& f = b->fields[i];
        if (f.d == c.d && f.n[0] == c.n[0] && f.n[1] == c.n[1] && f.n[2] == c.n[2]) mem.push_back(i);
      }
      std::sort(mem.begin(), mem.end(), [&](int64_t x, int64_t y) { return b->fields[x].stab_off < b->fields[y].stab_off; });
      b->class_order.insert(b->class_order.end(), mem.begin(), mem.end());
    }
  }
  sig << "|" << std::hex << hsh;
  b->signature = sig.str();
  b->twmax = twmax;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaMalloc(&b->tw, (size_t)(2 * twmax + kStageTableEntries) * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&b->stabs, (size_t)stab_total * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&b->ws, (size_t)ws_total * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&b->counters, (size_t)(3 * count + 2) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->outs, (size_t)count * sizeof(float*));
  if (e == cudaSuccess) e = cudaMalloc(&b->zouts, (size_t)count * sizeof(float*));
  if (e == cudaSuccess) e = cudaMalloc(&b->zfield, (size_t)count * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->seed_dev, sizeof(uint64_t));

  if (e == cudaSuccess)
    e = cudaMemcpy(b->zfield, b->class_order.data(), (size_t)count * sizeof(int64_t), cudaMemcpyHostToDevice);
  for (int q = 0; q < BatchPlan::kStreams && e == cudaSuccess; ++q) {
    e = cudaStreamCreateWithFlags(&b->cstreams[q], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->cjoin[q], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->cfork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = build_twiddles(b->tw, twmax, 0);
  for (int64_t i = 0; i < count && e == cudaSuccess; ++i) {
    const FieldInfo& f = b->fields[i];
    SpecParams sp{};
    sp.family = f.spec.family;
    sp.sigma = f.spec.sigma;
    sp.ell = f.spec.ell;
    sp.nu = f.spec.nu;
    sp.m = f.spec.m;
    sp.k = f.spec.k;
    sp.l = f.spec.l;
    sp.n = f.spec.n;
    sp.scale = 1.0;
    sp.d = f.d;
    for (int k = 0; k < 3; ++k) {
      sp.L[k] = f.L[k];
      sp.nn[k] = f.n[k];
    }
    e = build_stab(b->stabs + f.stab_off, nullptr, sp, 0.0, 0);
  }
  {  // s_k along k2 for the 1-D classes that take the four-step
    int64_t tot = 0;
    for (auto& c : b->classes)
      if (c.d == 1 && c.n[0] / 2 > 4096) {
        c.stabT_off = tot;
        tot += c.nf * (int64_t)(c.n[0] / 2);
      }
    if (e == cudaSuccess && tot) e = cudaMalloc(&b->stabsT, (size_t)tot * sizeof(float));
    for (const auto& c : b->classes) {
      if (e != cudaSuccess || c.stabT_off < 0) continue;
      const int M = c.n[0] / 2, lm = lg2(M);
      const int B = 1 << ((lm + 1) / 2), A = M / B;
      for (int64_t r = 0; r < c.nf && e == cudaSuccess; ++r)
        e = build_stab_fourstep(b->stabsT + c.stabT_off + r * M, b->stabs + c.stab_off + r * c.fold, A, B, 0);
    }
  }
  if (e == cudaSuccess) {
    std::vector<int> v;
    if (tune_cache_lookup(b->signature, &v) && v.size() == 2 && (v[0] == 128 || v[0] == 256) && v[1] >= 1 &&
        v[1] <= 4) {
      b->tile_threads = v[0];
      b->ctas_per_sm = v[1];
      b->tuned = true;
    }
    e = build_jobs(b);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    *err = std::string("batch plan: ") + cudaGetErrorString(e);
    batch_plan_free(b);
    return e == cudaErrorMemoryAllocation ? GRF_ERR_OOM : GRF_ERR_CUDA;
  }
  *out = b;
  return GRF_OK;
}

namespace {

// Per-shape mode: the seed goes to device memory (read by every launch), then
// the class launches, directly or from the graph captured for this output set.
grf_status sample_classes(BatchPlan* b, uint64_t seed, cudaStream_t s, bool use_graph, std::string* err) {
  cudaError_t e = cudaMemcpyAsync(b->seed_dev, &seed, sizeof(uint64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !use_graph) e = launch_classes(b, s);
  if (e == cudaSuccess && use_graph) {
    if (!b->cexec || b->cgraph_outs != b->cur_outs) {
      // this call's fields come from direct launches (which also set every
      // kernel's attributes outside the capture); the graph serves later calls
      e = launch_classes(b, s);
      if (e != cudaSuccess) {
        *err = std::string("batch launch: ") + cudaGetErrorString(e);
        return GRF_ERR_CUDA;
      }
      if (b->cexec) cudaGraphExecDestroy(b->cexec);
      if (b->cgraph) cudaGraphDestroy(b->cgraph);
      b->cexec = nullptr;
      b->cgraph = nullptr;
      cudaStream_t cs;
      e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the class streams are idle
      if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t le = launch_classes(b, cs);
        cudaError_t ce = cudaStreamEndCapture(cs, &b->cgraph);
        e = le != cudaSuccess ? le : ce;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->cexec, b->cgraph, 0);
      cudaStreamDestroy(cs);
      if (e != cudaSuccess) {
        if (b->cexec) cudaGraphExecDestroy(b->cexec);
        if (b->cgraph) cudaGraphDestroy(b->cgraph);
        b->cexec = nullptr;
        b->cgraph = nullptr;
        *err = std::string("batch graph capture: ") + cudaGetErrorString(e);
        return GRF_ERR_CUDA;
      }
      b->cgraph_outs = b->cur_outs;
      return GRF_OK;
    }
    e = cudaGraphLaunch(b->cexec, s);
  }
  if (e != cudaSuccess) {
    *err = std::string("batch launch: ") + cudaGetErrorString(e);
    return GRF_ERR_CUDA;
  }
  return GRF_OK;
}

}  // namespace

grf_status batch_plan_sample(BatchPlan* b, uint64_t seed, void* const* out, cudaStream_t s, int* status,
                             bool use_graph, std::string* err) {
  for (int64_t i = 0; i < b->count; ++i)
    if (!out[i]) {
      *err = "NULL output pointer";
      return GRF_ERR_INVALID_ARG;
    }
  cudaError_t e = set_outs(b, out, s);
  if (e != cudaSuccess) {
    *err = std::string("batch sample: ") + cudaGetErrorString(e);
    return GRF_ERR_CUDA;
  }
  b->status_dev = status;
  if (b->mode == 0 && b->withhold < 0) return sample_classes(b, seed, s, use_graph, err);
  if (e == cudaSuccess && !b->tuned) {
    const char* env = std::getenv("GRF_TUNE");
    if (!(env && env[0] == '0')) e = tune(b, seed, s, status);
    b->tuned = true;
  }
  if (e != cudaSuccess) {
    *err = std::string("batch sample: ") + cudaGetErrorString(e);
    return GRF_ERR_CUDA;
  }
  if (!use_graph) {
    e = launch_batch(b, seed, s, status);
    if (e != cudaSuccess) {
      *err = std::string("batch launch: ") + cudaGetErrorString(e);
      return GRF_ERR_CUDA;
    }
    return GRF_OK;
  }
  if (!b->exec || b->graph_outs != b->cur_outs) {
    drop_graph(b);
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the outs copy on s is complete
    if (e == cudaSuccess) e = prepare_kernel((const void*)batch_kernel, kBatchThreads, b->smem);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = launch_batch(b, seed, cs, status);
      cudaError_t ce = cudaStreamEndCapture(cs, &b->graph);
      e = le != cudaSuccess ? le : ce;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e == cudaSuccess) {
      size_t nn = 0;
      cudaGraphGetNodes(b->graph, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      cudaGraphGetNodes(b->graph, nodes.data(), &nn);
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) b->knode = nd;
      }
      if (!b->knode) e = cudaErrorUnknown;
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      drop_graph(b);
      *err = std::string("batch graph capture: ") + cudaGetErrorString(e);
      return GRF_ERR_CUDA;
    }
    b->graph_outs = b->cur_outs;
  }
  // the seed is a kernel parameter: set it on the instantiated graph, then replay
  BatchParams p = b->kparams;
  p.seed = seed;
  p.status = status;
  p.withhold_field = b->withhold;
  p.timeout_ns = b->timeout_ns;
  void* args[] = {&p};
  cudaKernelNodeParams kp{};
  e = cudaGraphKernelNodeGetParams(b->knode, &kp);
  if (e == cudaSuccess) {
    kp.kernelParams = args;
    kp.extra = nullptr;
    e = cudaGraphExecKernelNodeSetParams(b->exec, b->knode, &kp);
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) {
    *err = std::string("batch graph launch: ") + cudaGetErrorString(e);
    return GRF_ERR_CUDA;
  }
  return GRF_OK;
}

grf_status batch_plan_debug(BatchPlan* b, int withhold_field, double timeout_ms) {
  drop_graph(b);
  b->withhold = withhold_field;
  b->timeout_ns = timeout_ms > 0 ? (long long)(timeout_ms * 1e6) : kDefaultTimeoutNs;
  return GRF_OK;
}

int64_t batch_plan_total_points(const BatchPlan* b) { return b ? b->total_points : 0; }

grf_status batch_plan_set_mode(BatchPlan* b, int mode) {
  if (mode != 0 && mode != 1) return GRF_ERR_INVALID_ARG;
  b->mode = mode;
  return GRF_OK;
}

int batch_plan_mode(const BatchPlan* b) { return b ? b->mode : -1; }

void batch_plan_free(BatchPlan* b) {
  if (!b) return;
  drop_graph(b);
  if (b->cexec) cudaGraphExecDestroy(b->cexec);
  if (b->cgraph) cudaGraphDestroy(b->cgraph);
  for (int q = 0; q < BatchPlan::kStreams; ++q) {
    if (b->cstreams[q]) cudaStreamDestroy(b->cstreams[q]);
    if (b->cjoin[q]) cudaEventDestroy(b->cjoin[q]);
  }
  if (b->cfork) cudaEventDestroy(b->cfork);
  cudaFree(b->zouts);
  cudaFree(b->zfield);
  cudaFree(b->seed_dev);
  cudaFree(b->tw);
  cudaFree(b->stabs);
  cudaFree(b->stabsT);
  cudaFree(b->ws);
  cudaFree(b->jobs);
  cudaFree(b->items);
  cudaFree(b->counters);
  cudaFree(b->outs);
  delete b;
}

}  // namespace grf
