// Launchers of the FP32 passes of the sampling path, its Algorithm 1 mode and
// its adjoint (the kernels are in pass_kernels.cuh; the noise pass, compiled
// per noise variant, in noise_kernels.cu).
//
// Column pass (col_kernel): C consecutive columns of a plane, each a complex
// sequence along a strided axis.  With COL_NOISE it is the first pass of
// Algorithm 2 (§3): the kernel draws the Hermitian noise xi_K of every entry
// of its columns in registers (Philox4x32-10 + Box-Muller, the conjugate
// rule of Eq. conj on the planes k_d in {0, N_d/2}), multiplies by s_K
// (rule a) / Eq. drf) and runs the inverse FFT along axis 1; the noise never
// touches memory.  The last column pass before the c2r pass runs in pair mode
// and leaves Z of the c2r split (see col_body_pair).
//
// Row pass (row_kernel): C rows along the contiguous last axis.  ROW_C2R turns
// Z[0..M-1] into N = 2M reals with one M-point complex inverse FFT,
// z = IFFT_M(Z), f[2m] = Re z[m], f[2m+1] = Im z[m].  ROW_R2C is the forward
// counterpart (pack x[2m] + i x[2m+1], FFT_M, split).
#include <cstdlib>
#include "pass_kernels.cuh"

#include <mutex>

namespace grf {


// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

int points_per_thread(int n) { return n >= 16 ? 16 : n; }

// Pair mode adds one stash slot per point of the CTA (C N entries).
size_t col_pair_smem_bytes(int N, int C) { return col_smem_bytes(N, C) + (size_t)C * N * sizeof(float2); }

size_t col_smem_bytes(int N, int C) {
  size_t e = (size_t)spad_h(N) * C * sizeof(float2);
  const size_t red = 3 * sizeof(double) * 32;  // block_sum3 scratch
  return e > red ? e : red;
}

size_t row_smem_bytes(int M, int C) {
  size_t e = (size_t)(spad_h(M) + 1) * C * sizeof(float2);
  const size_t red = 3 * sizeof(double) * 1024;  // ROW_R2C_ADJ per-thread partials
  (void)red;
  return e;
}

// Shared-memory carveout: ask for what the resident CTAs need and leave the
// rest of the SM's 256 KB to L1, which holds the twiddle tables (a maximal
// carveout starves L1 and sends every twiddle load to L2).
cudaError_t prepare_kernel(const void* k, int threads, size_t smem) {
  struct Entry {
    const void* k;
    int threads;
    size_t smem;
  };
  // a fixed table (no host allocation on the launch path); when full, the
  // attributes are simply set again on every launch of an unseen configuration
  static std::mutex mu;
  static Entry done[512];
  static int ndone = 0;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < ndone; ++i)
    if (done[i].k == k && done[i].threads == threads && done[i].smem == smem) return cudaSuccess;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k);
  if (e != cudaSuccess) return e;
  const int regs = fa.numRegs > 0 ? fa.numRegs : 1;
  const int warps = (threads + 31) / 32;
  int blocks = 65536 / (warps * 32 * ((regs + 7) / 8 * 8));
  blocks = blocks < 1 ? 1 : blocks;
  blocks = blocks > 2048 / threads ? 2048 / threads : blocks;
  const size_t per = smem + fa.sharedSizeBytes + 1024;
  size_t need = per * blocks;
  const size_t cap = 228 * 1024;
  while (need > cap && blocks > 1) need = per * --blocks;
  int pct = (int)((need * 100 + cap - 1) / cap);
  pct = pct < 0 ? 0 : (pct > 100 ? 100 : pct);
  // the limit is a property of the kernel, not of the launch shape: raise it,
  // never lower it under a larger shape launched (and cached) before
  if (smem > 48 * 1024 && (int)smem > fa.maxDynamicSharedSizeBytes) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  if (e != cudaSuccess) return e;
  if (ndone < 512) done[ndone++] = Entry{k, threads, smem};
  return cudaSuccess;
}

template <int SRC, int MODE, int PAIR = 0>
static cudaError_t launch_col_p(int P, const ColArgs& a, dim3 grid, cudaStream_t s) {
  switch (P) {
    case 2: return launch_col_t<2, SRC, MODE, PAIR>(a, grid, s);
    case 4: return launch_col_t<4, SRC, MODE, PAIR>(a, grid, s);
    case 8: return launch_col_t<8, SRC, MODE, PAIR>(a, grid, s);
    case 16: return launch_col_t<16, SRC, MODE, PAIR>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_col(int src, int mode, int P, const ColArgs& a, dim3 grid, cudaStream_t s) {
  if (src == COL_NOISE && mode == COL_INV) return launch_col_noise(P, a, grid, s);
  cudaError_t e;
  if (src == COL_LOAD && mode == COL_INV && a.zpair && launch_col_load_pair_spec(P, a, grid, s, &e)) return e;
  if (a.zpair) {  // the inverse passes that end before the c2r pass
    if (src == COL_LOAD && mode == COL_INV) return launch_col_p<COL_LOAD, COL_INV, 1>(P, a, grid, s);
    if (src == COL_LOAD && mode == COL_FWD_SCALE_INV) return launch_col_p<COL_LOAD, COL_FWD_SCALE_INV, 1>(P, a, grid, s);
    return cudaErrorInvalidValue;
  }
  if (src == COL_LOAD && mode == COL_INV) return launch_col_p<COL_LOAD, COL_INV>(P, a, grid, s);
  if (src == COL_LOAD && mode == COL_FWD) return launch_col_p<COL_LOAD, COL_FWD>(P, a, grid, s);
  if (src == COL_LOAD && mode == COL_FWD_SCALE_INV) return launch_col_p<COL_LOAD, COL_FWD_SCALE_INV>(P, a, grid, s);
  if (src == COL_LOAD && mode == COL_FWD_ADJ) return launch_col_p<COL_LOAD, COL_FWD_ADJ>(P, a, grid, s);
  return cudaErrorInvalidValue;
}

template <int SRC, int MODE>
static cudaError_t launch_row_p(int P, const RowArgs& a, dim3 grid, cudaStream_t s) {
  switch (P) {
    case 1: return launch_row_t<1, SRC, MODE>(a, grid, s);
    case 2: return launch_row_t<2, SRC, MODE>(a, grid, s);
    case 4: return launch_row_t<4, SRC, MODE>(a, grid, s);
    case 8: return launch_row_t<8, SRC, MODE>(a, grid, s);
    case 16: return launch_row_t<16, SRC, MODE>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int P>
static cudaError_t launch_fourstep_t(int stage, const FourStepArgs& a, int64_t nfields, cudaStream_t s) {
  const int len = stage == 2 ? a.A : a.B;  // stages 1 and 3 transform along k2 (length B)
  const int ncols = stage == 2 ? a.B : a.A;
  const int threads = a.C * len / P;
  if (threads > 256) return cudaErrorInvalidValue;  // the kernels' launch bound
  const size_t smem = col_smem_bytes(len, a.C);
  const dim3 grid((unsigned)(ncols / a.C), 1, (unsigned)nfields);
  if (stage == 3) {  // stage 1 with mirror-closed columns: C / 2 column pairs per CTA
    const int H = a.C / 2;
    if (H < 1) return cudaErrorInvalidValue;
    auto k = fourstep_stage1_pair<P>;
    cudaError_t e = prepare_kernel((const void*)k, threads, smem);
    if (e != cudaSuccess) return e;
    k<<<dim3((unsigned)((a.A / 2 + 1 + H - 1) / H), 1, (unsigned)nfields), threads, smem, s>>>(a);
  } else if (stage == 1) {
    auto k = fourstep_stage1<P>;
    cudaError_t e = prepare_kernel((const void*)k, threads, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads, smem, s>>>(a);
  } else {
    auto k = fourstep_stage2<P>;
    cudaError_t e = prepare_kernel((const void*)k, threads, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_fourstep(int stage, int P, const FourStepArgs& a, int64_t nfields, cudaStream_t s) {
  if (P == 16 && std::getenv("GRF_FOURSTEP_GENERAL") == nullptr) {  // "GRF_FOURSTEP_GENERAL": run-time geometry only
    cudaError_t e = cudaSuccess;
    if (launch_fourstep_spec(stage, a, nfields, s, &e)) return e;
  }
  switch (P) {
    case 16: return launch_fourstep_t<16>(stage, a, nfields, s);
    default: return cudaErrorInvalidValue;  // both factors are >= 16
  }
}

template <int P>
static cudaError_t launch_row_gs_t(const RowArgs* ra, dim3 tiles, int ctas, cudaStream_t s) {
  const int threads = ra->C * (ra->M / P);
  const size_t smem = row_smem_bytes(ra->M, ra->C);
  auto k = row_kernel_gs<P, ROW_LOAD_Z, ROW_C2R>;
  cudaError_t e = prepare_kernel((const void*)k, threads, smem);
  if (e != cudaSuccess) return e;
  k<<<ctas, threads, smem, s>>>(*ra, (int64_t)tiles.x);
  return cudaGetLastError();
}

cudaError_t launch_row_c2r_gs(int P, const RowArgs& a, int64_t ntiles, int ctas, cudaStream_t s) {
  const dim3 t((unsigned)ntiles);
  switch (P) {
    case 1: return launch_row_gs_t<1>(&a, t, ctas, s);
    case 2: return launch_row_gs_t<2>(&a, t, ctas, s);
    case 4: return launch_row_gs_t<4>(&a, t, ctas, s);
    case 8: return launch_row_gs_t<8>(&a, t, ctas, s);
    case 16: return launch_row_gs_t<16>(&a, t, ctas, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_row(int src, int mode, int P, const RowArgs& a, dim3 grid, cudaStream_t s) {
  if (src == ROW_LOAD_Z && mode == ROW_C2R) {
    cudaError_t e;
    if (launch_row_c2r_spec(P, a, grid, s, &e)) return e;
    return launch_row_p<ROW_LOAD_Z, ROW_C2R>(P, a, grid, s);
  }
  if (src == ROW_NOISE_H && mode == ROW_C2R) return launch_row_p<ROW_NOISE_H, ROW_C2R>(P, a, grid, s);
  if (src == ROW_LOAD_REAL && mode == ROW_R2C) return launch_row_p<ROW_LOAD_REAL, ROW_R2C>(P, a, grid, s);
  if (src == ROW_NOISE_REAL && mode == ROW_R2C) return launch_row_p<ROW_NOISE_REAL, ROW_R2C>(P, a, grid, s);
  if (src == ROW_NOISE_REAL && mode == ROW_R2C_SCALE_C2R)
    return launch_row_p<ROW_NOISE_REAL, ROW_R2C_SCALE_C2R>(P, a, grid, s);
  if (src == ROW_LOAD_REAL && mode == ROW_R2C_ADJ) return launch_row_p<ROW_LOAD_REAL, ROW_R2C_ADJ>(P, a, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace grf
