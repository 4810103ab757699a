// The line kernel of the Neumann / Dirichlet fields (r2r.cu has the
// launchers; r2r_spec.cu the compile-time geometries).
#pragma once
#include "kernels.h"
#include "fft_core.cuh"

namespace grf {
namespace r2r {


constexpr int kR2rThreads = 512;
constexpr bool kR2rPrefetch = false;  // twiddles loaded after each exchange: fewer spills at 64 registers
constexpr int kR2rMinBlocks = 2;  // 64 registers: two 512-thread CTAs per SM (measured 1.4x over one)

constexpr int64_t kFaceLine = int64_t(1) << 62;

// Offset of point 0 of line lg (over the whole batch), or -1 past the end.
// Dirichlet: kFaceLine is added for a line on a face of another axis (a
// coordinate 0 or N_i there), which is written as exact zeros: computed, it
// would carry the rounding residue of its partner line.
GRF_DEV int64_t r2r_line_base(const R2rArgs& a, int64_t lg) {
  if (lg >= a.nlines) return -1;
  const int64_t b = lg / a.lines_per_field;
  const int64_t r = lg - b * a.lines_per_field;
  const int64_t o = r / a.inner;
  const int64_t i = r - o * a.inner;
  int64_t base = b * a.field_stride + o * (int64_t)(a.N + 1) * a.inner + i;
  if (a.bc == 2) {
    bool face = false;
    int64_t rem = i;
    for (int x = a.d - 1; x > a.axis; --x) {
      const int64_t cx = rem % a.pts[x];
      rem /= a.pts[x];
      face |= cx == 0 || cx == a.pts[x] - 1;
    }
    rem = o;
    for (int x = a.axis - 1; x >= 0; --x) {
      const int64_t cx = rem % a.pts[x];
      rem /= a.pts[x];
      face |= cx == 0 || cx == a.pts[x] - 1;
    }
    if (face) base += kFaceLine;
  }
  return base;
}

// SRC: where the lines come from (compile time, so that each kernel holds
// only the code it runs); BC: 1 Neumann, 2 Dirichlet; LNF, CC != 0: the
// transform length 2N = 2^LNF and CC line pairs per CTA as constants (the
// stage loop unrolls, exchange and twiddle addresses become constant
// offsets, and the divisions by the line length become multiplications).
enum R2rSrc { R2R_NOISE_ROWS = 0, R2R_LOAD_ROWS = 1, R2R_LOAD_STRIDED = 2 };

template <int P, int SRC, int BC, int LNF = 0, int CC = 0>
__global__ void __launch_bounds__(kR2rThreads, kR2rMinBlocks) r2r_line_kernel(R2rArgs a) {
  extern __shared__ float2 sm[];
  constexpr bool spec = LNF && CC;
  const int C = spec ? CC : a.C;
  const int logC = spec ? ilog2c(CC) : a.logC;
  const int G = 2 * C;
  const int N = spec ? (1 << (LNF - 1)) : a.N;
  const int NF = 2 * N;
  const int logNF = spec ? LNF : a.logNF;
  const int logG = logC + 1;
  const int TPT = NF / P;
  const int nthr = C * TPT;
  const int t = threadIdx.x;
  const int c = t & (C - 1);
  const int tau = t >> logC;
  const int64_t l0 = (int64_t)blockIdx.x * G;
  // the tile of the CTA's lines: rows (contiguous lines) line-major, point n of
  // line l at l W + n; strided lines point-major, at n G + l (G = 2C lines)
  float* tile = reinterpret_cast<float*>(sm);
  const int W = N + 1;
  int64_t* lbase = reinterpret_cast<int64_t*>(sm + (size_t)spad(NF) * C);
  int64_t* lj0 = lbase + G;  // noise launch: flat index of point 0 of each line in its field
  uint64_t* lkey = reinterpret_cast<uint64_t*>(lj0 + G);  // and the Philox key of its field
  constexpr bool dirichlet = BC == 2;

  for (int l = t; l < G; l += nthr) {
    const int64_t base = r2r_line_base(a, l0 + l);
    lbase[l] = base;
    if constexpr (SRC == R2R_NOISE_ROWS) {
      if (base >= 0) {
        const int64_t b = (l0 + l) / a.lines_per_field;
        lj0[l] = (base & (kFaceLine - 1)) - b * a.field_stride;
        lkey[l] = a.seed + (uint64_t)(a.field0 + b);
      }
    }
  }
  __syncthreads();

  // 1. the CTA's lines into the tile
  if constexpr (SRC == R2R_NOISE_ROWS) {  // rows of the last axis: a_K t_K, four points per Philox call
    const int NQ = (N + 3) / 4 + 1;  // calls that can touch one row of N + 1 points
    for (int u = t; u < G * NQ; u += nthr) {
      const int l = u / NQ;
      const int qi = u - l * NQ;
      const int64_t base = lbase[l];
      if (base < 0 || base >= kFaceLine) {
        for (int n = qi; n <= N; n += NQ) tile[l * W + n] = 0.f;
        continue;
      }
      const int64_t j0 = lj0[l];
      const int64_t m = (j0 >> 2) + qi;
      const int d = (int)(4 * m - j0);  // position in the line of the call's first point, -3..N + 3
      if (d > N) continue;
      const u32x4 w = philox_call((uint64_t)m, 2u, lkey[l]);
      const float2 z01 = box_muller(w.x, w.y, a.trig);
      const float2 z23 = box_muller(w.z, w.w, a.trig);
      const float z[4] = {z01.x, z01.y, z23.x, z23.y};
      const float* tb = a.tab + 4 * m;  // t_K of the call's points
      const int row = l * W + d;
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (d + s >= 0 && d + s <= N) tile[row + s] = z[s] * __ldg(tb + s);
    }
  } else if constexpr (SRC == R2R_LOAD_ROWS) {  // contiguous rows
    for (int e = t; e < W * G; e += nthr) {
      const int l = e / W;
      const int n = e - l * W;
      const int64_t base = lbase[l];
      tile[e] = (base >= 0 && base < kFaceLine) ? __ldcg(a.f + base + n) : 0.f;
    }
  } else {  // strided axis: neighbouring lines are neighbours in memory;
            // sixteen loads in flight per thread before they go to the tile
    const int E = W * G;
    constexpr int U = 16;
    for (int e0 = t; e0 < E; e0 += U * nthr) {
      float x[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * nthr;
        x[u] = 0.f;
        if (e < E) {
          const int64_t base = lbase[e & (G - 1)];
          if (base >= 0 && base < kFaceLine) x[u] = __ldcg(a.f + base + (int64_t)(e >> logG) * a.inner);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (e0 + u * nthr < E) tile[e0 + u * nthr] = x[u];
    }
  }
  cta_sync(nthr);

  // 2. the even / odd extension of the pair (2c, 2c + 1), length 2N
  const float2* tile2 = reinterpret_cast<const float2*>(sm);
  float2 v[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int n = tau + TPT * q;
    const int nn = n <= N ? n : NF - n;
    float2 x;
    if constexpr (SRC == R2R_LOAD_STRIDED) x = tile2[nn * C + c];
    else x = make_float2(tile[2 * c * W + nn], tile[(2 * c + 1) * W + nn]);
    if (dirichlet) {
      if (n == 0 || n == N) x = make_float2(0.f, 0.f);
      else if (n > N) x = make_float2(-x.x, -x.y);
    }
    v[q] = x;
  }
  fft_core<P, +1, kR2rPrefetch>(v, sm, tau, c, C, NF, logNF, a.tw, a.tws, nthr);

  // 3. outputs 0..N, separated into the two lines
  cta_sync(nthr);
  float2* out2 = reinterpret_cast<float2*>(sm);
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int k = tau + TPT * q;
    if (k <= N) {
      const float2 y = v[q];
      float2 o = y;
      if (dirichlet) o = (k == 0 || k == N) ? make_float2(0.f, 0.f) : make_float2(y.y, -y.x);
      if constexpr (SRC == R2R_LOAD_STRIDED) {
        out2[k * C + c] = o;
      } else {
        tile[2 * c * W + k] = o.x;
        tile[(2 * c + 1) * W + k] = o.y;
      }
    }
  }
  cta_sync(nthr);

  // 4. the tile back to global memory, as it was read
  if constexpr (SRC != R2R_LOAD_STRIDED) {
    for (int l = 0; l < G; ++l) {  // line by line: no division, one base per line
      const int64_t base = lbase[l];
      if (base < 0) continue;
      float* dst = a.f + (base & (kFaceLine - 1));
      const float* src = tile + l * W;
      const bool face = base >= kFaceLine;
      for (int n = t; n < W; n += nthr) dst[n] = face ? 0.f : src[n];
    }
  } else {
    const int E = W * G;
    for (int e = t; e < E; e += nthr) {
      const int n = e >> logG;
      const int l = e & (G - 1);
      const int64_t base = lbase[l];
      if (base >= 0) a.f[(base & (kFaceLine - 1)) + (int64_t)n * a.inner] = base < kFaceLine ? tile[e] : 0.f;
    }
  }
}

template <int P, int SRC, int BC, int LNF = 0, int CC = 0>
cudaError_t launch_r2r_t(const R2rArgs& a, cudaStream_t s) {
  const int threads = a.C * (2 * a.N / P);
  const size_t smem = r2r_smem_bytes(a.N, a.C);
  const int64_t ctas = (a.nlines + 2 * a.C - 1) / (2 * a.C);
  if (ctas > 0x7FFFFFFF) return cudaErrorInvalidValue;
  auto k = r2r_line_kernel<P, SRC, BC, LNF, CC>;
  cudaError_t e = prepare_kernel((const void*)k, threads, smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)ctas, threads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace r2r

// The compile-time geometries (r2r_spec.cu): true if one matched and was
// launched (its status in *err).
bool launch_r2r_spec(int src, const R2rArgs& a, cudaStream_t s, cudaError_t* err);

}  // namespace grf
