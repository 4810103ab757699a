// Neumann and Dirichlet fields (the cosine / sine transform variant that §1
// and §3 mention): on the box [0, L_i] with N_i intervals per axis,
//   f_J = sum_K t_K a_K prod_i E(k_i, j_i),  J, K in prod{0..N_i},
// E = cos(pi k j / N) (Neumann) or sin(pi k j / N) (Dirichlet), a_K real
// normals, t_K from the spectral density on the mirrored box of edges 2 L_i.
//
// One kernel, one launch per axis, in place on the caller's output: a CTA
// takes 2C lines of one axis (N + 1 points each), packs lines 2c and 2c + 1
// into one complex sequence x_a + i x_b, extends it evenly (Neumann: z_n =
// z_{2N-n}) or oddly (Dirichlet: z_{2N-n} = -z_n, z_0 = z_N = 0) to length 2N,
// runs one inverse FFT of length 2N, and keeps outputs 0..N.  For real even
// (odd) data the transform is real (imaginary), so the two lines separate:
//   Neumann:   y = e_0 + (-1)^j e_N + 2 sum_{0<n<N} e_n cos(pi n j / N)  -> (Re, Im)
//   Dirichlet: y = 2 sum_{0<n<N} e_n sin(pi n j / N)                     -> (Im, -Re)
// The factor 2 on interior coefficients is the extension's, so the table
// holds t_K = sqrt(w_K S(p_K) / |2D|) / 2^(number of interior k_i).
// The first launch (the last axis, contiguous rows) draws a_K itself, with
// the flat index j of K: call j >> 2, counter (q_lo, q_hi, 2, 0), words 2t,
// 2t + 1 (t = (j & 3) >> 1), even j the cosine normal, odd j the sine normal.
// Each line is staged through shared memory between global memory and the
// FFT's register layout, so that global loads and stores are coalesced along
// whichever direction is contiguous: along the points of a row, or across
// neighbouring lines of a strided axis.
#include "kernels.h"
#include "fft_core.cuh"

namespace grf {

namespace {

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
// only the code it runs); BC: 1 Neumann, 2 Dirichlet.
enum R2rSrc { R2R_NOISE_ROWS = 0, R2R_LOAD_ROWS = 1, R2R_LOAD_STRIDED = 2 };

template <int P, int SRC, int BC>
__global__ void __launch_bounds__(kR2rThreads, kR2rMinBlocks) r2r_line_kernel(R2rArgs a) {
  extern __shared__ float2 sm[];
  const int C = a.C;
  const int G = 2 * C;
  const int N = a.N;
  const int NF = 2 * N;
  const int TPT = NF / P;
  const int nthr = C * TPT;
  const int t = threadIdx.x;
  const int c = t & (C - 1);
  const int tau = t >> a.logC;
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
      if (4 * m > j0 + N) continue;
      const u32x4 w = philox_call((uint64_t)m, 2u, lkey[l]);
      const float2 z01 = box_muller(w.x, w.y, a.trig);
      const float2 z23 = box_muller(w.z, w.w, a.trig);
      const float z[4] = {z01.x, z01.y, z23.x, z23.y};
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int64_t j = 4 * m + s;
        if (j >= j0 && j <= j0 + N) tile[l * W + (int)(j - j0)] = z[s] * __ldg(a.tab + j);
      }
    }
  } else if constexpr (SRC == R2R_LOAD_ROWS) {  // contiguous rows
    for (int e = t; e < W * G; e += nthr) {
      const int l = e / W;
      const int n = e - l * W;
      const int64_t base = lbase[l];
      tile[e] = (base >= 0 && base < kFaceLine) ? __ldcg(a.f + base + n) : 0.f;
    }
  } else {  // strided axis: neighbouring lines are neighbours in memory;
            // eight loads in flight per thread before they go to the tile
    const int E = W * G;
    constexpr int U = 8;
    for (int e0 = t; e0 < E; e0 += U * nthr) {
      float x[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * nthr;
        x[u] = 0.f;
        if (e < E) {
          const int64_t base = lbase[e & (G - 1)];
          if (base >= 0 && base < kFaceLine) x[u] = __ldcg(a.f + base + (int64_t)(e >> a.logG) * a.inner);
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
  fft_core<P, +1, kR2rPrefetch>(v, sm, tau, c, C, NF, a.logNF, a.tw, a.tws, nthr);

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
    for (int e = t; e < W * G; e += nthr) {
      const int l = e / W;
      const int n = e - l * W;
      const int64_t base = lbase[l];
      if (base >= 0) a.f[(base & (kFaceLine - 1)) + n] = base < kFaceLine ? tile[e] : 0.f;
    }
  } else {
    const int E = W * G;
    for (int e = t; e < E; e += nthr) {
      const int n = e >> a.logG;
      const int l = e & (G - 1);
      const int64_t base = lbase[l];
      if (base >= 0) a.f[(base & (kFaceLine - 1)) + (int64_t)n * a.inner] = base < kFaceLine ? tile[e] : 0.f;
    }
  }
}

template <int P, int SRC, int BC>
cudaError_t launch_r2r_t(const R2rArgs& a, cudaStream_t s) {
  const int threads = a.C * (2 * a.N / P);
  const size_t smem = r2r_smem_bytes(a.N, a.C);
  const int64_t ctas = (a.nlines + 2 * a.C - 1) / (2 * a.C);
  if (ctas > 0x7FFFFFFF) return cudaErrorInvalidValue;
  auto k = r2r_line_kernel<P, SRC, BC>;
  cudaError_t e = prepare_kernel((const void*)k, threads, smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)ctas, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_r2r_p(int src, const R2rArgs& a, cudaStream_t s) {
  const bool dir = a.bc == 2;
  switch (src) {
    case R2R_NOISE_ROWS: return dir ? launch_r2r_t<P, R2R_NOISE_ROWS, 2>(a, s) : launch_r2r_t<P, R2R_NOISE_ROWS, 1>(a, s);
    case R2R_LOAD_ROWS: return dir ? launch_r2r_t<P, R2R_LOAD_ROWS, 2>(a, s) : launch_r2r_t<P, R2R_LOAD_ROWS, 1>(a, s);
    default: return dir ? launch_r2r_t<P, R2R_LOAD_STRIDED, 2>(a, s) : launch_r2r_t<P, R2R_LOAD_STRIDED, 1>(a, s);
  }
}

}  // namespace

// FFT scratch (which also holds the tile), then per line: the offset of point
// 0, and for the noise launch its flat index in the field and its Philox key
size_t r2r_smem_bytes(int N, int C) { return (size_t)spad_h(2 * N) * C * sizeof(float2) + 3 * 2 * C * sizeof(int64_t); }

int r2r_points_per_thread(int N) { return 2 * N >= 16 ? 16 : 2 * N; }

int r2r_lines_per_cta(int N) {
  const int TPT = 2 * N / r2r_points_per_thread(N);
  int C = kR2rThreads / TPT;
  if (C > 256) C = 256;
  return C < 1 ? 1 : C;
}

cudaError_t launch_r2r(const R2rArgs& a, cudaStream_t s) {
  if (a.N < 2 || (a.N & (a.N - 1)) || a.N > 4096 || a.C < 1 || (a.C & (a.C - 1))) return cudaErrorInvalidValue;
  if (a.C * (2 * a.N / r2r_points_per_thread(a.N)) > kR2rThreads) return cudaErrorInvalidValue;
  if (a.noise && a.inner != 1) return cudaErrorInvalidValue;
  const int src = a.noise ? R2R_NOISE_ROWS : (a.inner == 1 ? R2R_LOAD_ROWS : R2R_LOAD_STRIDED);
  switch (r2r_points_per_thread(a.N)) {
    case 4: return launch_r2r_p<4>(src, a, s);
    case 8: return launch_r2r_p<8>(src, a, s);
    case 16: return launch_r2r_p<16>(src, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace grf
