// Shared-memory Stockham stages of any radix in {2, 3, 4, 5, 7, 8}, for the
// fused passes of FP32 2-D grids whose sizes are 2^a 3^b 5^c 7^d (mixed_fused.cu).
//
// A stage of radix R and span Ns over sequences of length N (Ns R divides N):
// butterfly j < N / R reads positions j + r N / R, multiplies input r by
// e^{2 pi i (j mod Ns) r / (R Ns)}, takes the inverse DFT of R points and writes
// position (j - j mod Ns) R + j mod Ns + r Ns (Stockham autosort: after the
// last stage the sequence is in natural order, whatever the order of radices).
// Twiddles come from a per-length stage table (FP64-built, mixed_fused.cu).
#pragma once
#include "fft_core.cuh"

namespace grf {

// cos and sin of 2 pi j / R for R = 3, 5, 7 and j = 1 .. (R - 1) / 2.
__host__ __device__ constexpr double cos_2pi(int R, int j) {
  return R == 3 ? -0.5
       : R == 5 ? (j == 1 ? 0.30901699437494742410 : -0.80901699437494742410)
                : (j == 1 ? 0.62348980185873353053 : j == 2 ? -0.22252093395631440429 : -0.90096886790241912624);
}
__host__ __device__ constexpr double sin_2pi(int R, int j) {
  return R == 3 ? 0.86602540378443864676
       : R == 5 ? (j == 1 ? 0.95105651629515357212 : 0.58778525229247312917)
                : (j == 1 ? 0.78183148246802980871 : j == 2 ? 0.97492791218182360702 : 0.43388373911755812048);
}

// Inverse DFT of an odd number R of points in place:
// X[k] = x0 + sum_n (x[n] + x[R-n]) cos(2 pi n k / R) + i (x[n] - x[R-n]) sin(2 pi n k / R),
// X[R - k] the same with -i.
template <int R>
GRF_DEV void dft_odd(float2 (&x)[R]) {
  constexpr int h = (R - 1) / 2;
  float2 a[h], b[h];
#pragma unroll
  for (int n = 1; n <= h; ++n) {
    a[n - 1] = cadd(x[n], x[R - n]);
    b[n - 1] = csub(x[n], x[R - n]);
  }
  const float2 x0 = x[0];
  float2 s0 = x0;
#pragma unroll
  for (int n = 0; n < h; ++n) s0 = cadd(s0, a[n]);
#pragma unroll
  for (int k = 1; k <= h; ++k) {
    float2 ar = x0, bi = make_float2(0.f, 0.f);
#pragma unroll
    for (int n = 1; n <= h; ++n) {
      const int j = (n * k) % R;  // angle 2 pi j / R
      const int jj = j <= h ? j : R - j;
      const float sg = j <= h ? 1.f : -1.f;
      const float c = (float)cos_2pi(R, jj);
      const float s = sg * (float)sin_2pi(R, jj);
      ar = make_float2(fmaf(a[n - 1].x, c, ar.x), fmaf(a[n - 1].y, c, ar.y));
      bi = make_float2(fmaf(b[n - 1].x, s, bi.x), fmaf(b[n - 1].y, s, bi.y));
    }
    // X[k] = ar + i bi, X[R - k] = ar - i bi
    x[k] = make_float2(ar.x - bi.y, ar.y + bi.x);
    x[R - k] = make_float2(ar.x + bi.y, ar.y - bi.x);
  }
  x[0] = s0;
}

template <int R>
GRF_DEV void dft_small(float2 (&x)[R]) {
  if constexpr (R == 2 || R == 4 || R == 8) dft_regs<R, +1, 1, 0>(x);
  else dft_odd<R>(x);
}

// floor(n / d) for 0 <= n < 2^22 from rd = the correctly rounded 1 / d: the
// product (n + 1/2) rd is within 2^-23 (n + 1/2) / d of (n + 1/2) / d, less
// than the 1 / (2d) that separates (n + 1/2) / d from the nearest integer.
GRF_DEV int qdiv(int n, float rd) { return __float2int_rz(((float)n + 0.5f) * rd); }

// One stage over C sequences of length N (sequence c at src + c * pitch), by
// the nthr threads t < nthr; the caller synchronises around it.  The stage's
// twiddles e^{2 pi i m r / (R Ns)} sit at tab[Ns - 1 + (r - 1) Ns + m]: lanes
// with consecutive m read consecutive entries.
template <int R>
GRF_DEV void mixed_stage(const float2* __restrict__ src, float2* __restrict__ dst, int pitch, int N, int Ns, int C,
                         const float2* __restrict__ tab, int t, int nthr) {
  const int nb = N / R;
  const float rnb = __frcp_rn((float)nb), rNs = __frcp_rn((float)Ns);
  for (int idx = t; idx < C * nb; idx += nthr) {
    const int c = C == 1 ? 0 : qdiv(idx, rnb);
    const int j = idx - c * nb;
    const int q = qdiv(j, rNs);
    const int m = j - q * Ns;
    const float2* s = src + c * pitch;
    float2* d = dst + c * pitch;
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = s[j + r * nb];
    if (Ns > 1) {
      const float2* w = tab + (Ns - 1) + m;
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = cmul(x[r], __ldg(w + (r - 1) * Ns));
    }
    dft_small<R>(x);
    const int base = q * Ns * R + m;
#pragma unroll
    for (int r = 0; r < R; ++r) d[base + r * Ns] = x[r];
  }
}

// All stages of the inverse DFT of C sequences of length N held in buffer a
// (pitch `pitch`), ping-ponging with buffer b; returns the buffer that holds
// the result.  radix[0..nst) multiply to N; tab is the length's stage table.
// Starts and ends with a barrier over the whole CTA.
GRF_DEV float2* mixed_transform(float2* a, float2* b, int pitch, int N, int C, const int* radix, int nst,
                                const float2* __restrict__ tab) {
  const int t = threadIdx.x, nthr = blockDim.x;
  int Ns = 1;
  for (int st = 0; st < nst; ++st) {
    __syncthreads();
    switch (radix[st]) {
      case 2: mixed_stage<2>(a, b, pitch, N, Ns, C, tab, t, nthr); break;
      case 3: mixed_stage<3>(a, b, pitch, N, Ns, C, tab, t, nthr); break;
      case 4: mixed_stage<4>(a, b, pitch, N, Ns, C, tab, t, nthr); break;
      case 5: mixed_stage<5>(a, b, pitch, N, Ns, C, tab, t, nthr); break;
      case 7: mixed_stage<7>(a, b, pitch, N, Ns, C, tab, t, nthr); break;
      default: mixed_stage<8>(a, b, pitch, N, Ns, C, tab, t, nthr); break;
    }
    Ns *= radix[st];
    float2* x = a;
    a = b;
    b = x;
  }
  __syncthreads();
  return a;
}

}  // namespace grf
