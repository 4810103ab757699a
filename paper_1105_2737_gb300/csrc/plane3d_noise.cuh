// Pass 1 of the 3-D plane path (see PlaneArgs in kernels.h): Philox noise,
// the Hermitian arrangement (Lemma 1; Eq. conj on the planes k3 in {0, M}) and
// s_K in registers, the inverse FFT along axis 1, then the first radix-R step
// of the inverse FFT along axis 2, written as R independent sub-planes.
//
// A CTA (256 threads, CC = 4096 / N1 columns of length N1) takes the columns
// (k2 = k' + Q r, k3 = k3_0 + u) for r < R and u < U = CC / R, k' = blockIdx.y,
// k3_0 = U blockIdx.x; column c = r U + u.  After the axis-1 transforms the
// columns go through shared memory ([c][j1], pitch N1 + 1) so that each thread
// holds the R values X[j1, k' + Q r, k3] of one (j1, u) and forms
//   B_s = w^{k' s} sum_r X_r e^{2 pi i r s / R},  s < R,  w = e^{2 pi i / N2}
// (decimation in frequency: the length-N2 inverse DFT then splits into R
// inverse DFTs of length Q over k', one per residue s of j2 mod R).
#pragma once
#include "noise_fast.cuh"

namespace grf {

// Shared memory: the transform's exchange buffer (also the [c][j1] staging of
// the radix-R step: CC (N1 + 1) <= CC spad(N1)) and the 256 coarse angles.
__host__ __device__ constexpr size_t plane3_noise_smem_bytes(int N1, int CC) {
  return ((size_t)(N1 + N1 / 16) * CC + 256) * sizeof(float2);
}

template <int LN, int CC, int R>
__global__ void __launch_bounds__(256, 3) plane3_noise_kernel(ColArgs a, PlaneArgs pl) {
  // The staged columns sit at slot (c mod U) R + c / U with a pitch of N + 16 / CC
  // float2: a half warp's 64-bit accesses then fall on 16 distinct bank pairs
  // both when it writes (16 / CC rows of all CC columns) and when it reads the
  // radix-R inputs (16 / U rows of U consecutive k3).
  constexpr int P = 16, N = 1 << LN, TPT = N / P, NTHR = CC * TPT, U = CC / R, PITCH = N + 16 / CC;
  static_assert(NTHR == 256 && CC % R == 0, "256-thread geometries, R dividing the columns per CTA");
  extern __shared__ float2 sm[];
  float2* strig = sm + (size_t)(N + N / 16) * CC;
  const HalfGeom& g = a.g;
  strig[CtaCoordsHW{}.tid()] = __ldg(g.trig + CtaCoordsHW{}.tid());
  __syncthreads();

  const int M = g.M, N2 = pl.N2, Q = pl.Q;
  const uint64_t key = field_key(g, blockIdx.z);  // uniform
  const int kp = blockIdx.y;
  float2 v[P];
  {
    const int t = CtaCoordsHW{}.tid();
    const int c = t & (CC - 1), tau = t / CC;
    const int r = c / U, u = c - (c / U) * U;
    const int k2 = kp + Q * r;
    const int k3 = (int)blockIdx.x * U + u;
    const bool valid = k3 <= M;
    const int kd = valid ? k3 : 0;
    const float* srow = field_stab(g, blockIdx.z) + ((size_t)kd * (N2 / 2 + 1) + min(k2, N2 - k2)) * (N / 2 + 1);
    if (kd != 0 && kd != M) {
      normals_half<P, TPT>(v, tau, k2, kd, N2, M, key, strig);
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const float s = __ldg(srow + (q < P / 2 ? tau + TPT * q : N - tau - TPT * q));
        v[q] = cscale(v[q], s);
      }
    } else {
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const float s = __ldg(srow + (q < P / 2 ? tau + TPT * q : N - tau - TPT * q));
        v[q] = cscale(plane_xi(tau + TPT * q, k2, kd, N, N2, M, key, g.trig), s);
      }
    }
    if (!valid) {
#pragma unroll
      for (int q = 0; q < P; ++q) v[q] = make_float2(0.f, 0.f);
    }
    fft_core<P, +1>(v, sm, tau, c, CC, N, LN, a.tw, a.tws, NTHR);
  }
  __syncthreads();  // the transform's last exchange has been read by every thread
  {
    const int t = CtaCoordsHW{}.tid();
    const int c = t & (CC - 1), tau = t / CC;
    const int slot = (c % U) * R + c / U;
#pragma unroll
    for (int q = 0; q < P; ++q) sm[slot * PITCH + tau + TPT * q] = v[q];
  }
  __syncthreads();

  // the radix-R step: items (j1, u), u fastest (U consecutive k3 per store run)
  const float2* tw2 = pl.tw + N2;  // exp(2 pi i k / N2)
  const int S3 = pl.S3;
  float2* wsf = pl.ws + (int64_t)blockIdx.z * ((int64_t)N * N2 * S3);
  constexpr int ITEMS = N * U / NTHR;
  const int t = CtaCoordsHW{}.tid();
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int i = it * NTHR + t;
    const int j1 = i / U, u = i - (i / U) * U;
    const int k3 = (int)blockIdx.x * U + u;
    if (k3 > M) continue;
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = sm[(u * R + r) * PITCH + j1];
    dft_regs<R, +1, 1, 0>(x);  // x[s] = sum_r X_r e^{+2 pi i r s / R}
    float2* dst = wsf + ((int64_t)j1 * R * Q + kp) * S3 + k3;
#pragma unroll
    for (int s = 0; s < R; ++s) dst[(int64_t)s * Q * S3] = s ? cmul(x[s], __ldg(tw2 + kp * s)) : x[s];
  }
}

}  // namespace grf
