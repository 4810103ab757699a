// Device helpers shared by the GRF kernels: complex arithmetic, the
// Philox4x32-10 counter-based generator and the Box-Muller transform.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define GRF_DEV __device__ __forceinline__

namespace grf {

GRF_DEV float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
GRF_DEV float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
GRF_DEV float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
GRF_DEV float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
GRF_DEV float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
GRF_DEV float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

GRF_DEV double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
GRF_DEV double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
GRF_DEV double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
GRF_DEV double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
GRF_DEV double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
//   c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
// with the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct u32x4 {
  uint32_t x, y, z, w;
};

GRF_DEV u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                            uint32_t k1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t lo0 = M0 * c0, hi0 = __umulhi(M0, c0);
    const uint32_t lo1 = M1 * c2, hi1 = __umulhi(M1, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return u32x4{c0, c1, c2, c3};
}

// Call q (64-bit) with counter (q_lo, q_hi, tag, 0) and key (lo, hi) of `key`.
GRF_DEV u32x4 philox_call(uint64_t q, uint32_t tag, uint64_t key) {
  return philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), tag, 0u, (uint32_t)key,
                       (uint32_t)(key >> 32));
}

// u = (2 (x >> 9) + 1) 2^-24: exact in FP32, in (0, 1).  Formed from the bits:
// the float with exponent 0 and mantissa x >> 9 is 1 + (x >> 9) 2^-23, and adding
// 2^-24 - 1 (exact in FP32) gives u, which is representable, so the add is exact.
GRF_DEV float uniform_open(uint32_t x) {
  return __int_as_float(0x3F800000u | (x >> 9)) + (-0.999999940395355224609375f);
}
GRF_DEV double uniform_open_d(uint32_t x) {
  return (double)((x >> 9) * 2u + 1u) * 5.9604644775390625e-8;
}

// Box-Muller: rho = sqrt(-2 ln u_a), (z_re, z_im) = rho (cos 2 pi u_b, sin 2 pi u_b).
// ln u_a: CUDA's fast __logf, whose error is at most 3 ulp for u < 0.5 and at
// most 2^-21.41 absolute on [0.5, 2); within 2^-7 of 1, where that bound would
// be large against |ln u|, the series ln(1 - t) = -(t + t^2/2 + t^3/3 + t^4/4)
// (truncation below 2^-28 relative) on t = 1 - u, which is exact (Sterbenz).
// Both are formed and one is selected, without a branch.
// The angle: u_b = m' 2^-24 with m' = 2 (x >> 9) + 1
// an odd 24-bit integer, so 2 pi u_b = a + delta exactly, with the coarse angle
// a = 2 pi (m' >> 16) / 256 and delta = 2 pi (m' & 0xFFFF) 2^-24 in [0, 0.0246).
// cos a, sin a come from `trig` (trig[h] = exp(2 pi i h / 256), built in FP64);
// cos delta, sin delta from their Taylor series (truncation below 4e-13), and the
// angle-addition formulas combine them.  Error: a few FP32 ulps.
GRF_DEV float2 box_muller(uint32_t wa, uint32_t wb, const float2* __restrict__ trig) {
  const float ua = uniform_open(wa);
  const float ta = 1.0f - ua;
  const float near1 = -ta * fmaf(ta, fmaf(ta, fmaf(ta, 0.25f, 0.333333343f), 0.5f), 1.0f);
  const float rho2 = -2.0f * (ta < 0.0078125f ? near1 : __logf(ua));
  const float rho = rho2 * rsqrtf(rho2);
  // m' >> 16 = wb >> 24; m' & 0xFFFF = 2 r + 1 with r = (wb >> 9) & 0x7FFF, and
  // (2 r + 1) 2^-16 is formed exactly from the bits as in uniform_open, then
  // scaled by 2 pi / 2^8 (the same product as (2 r + 1) times 2 pi / 2^24)
  const float2 t = __ldg(trig + (wb >> 24));
  const float dl = (__int_as_float(0x3F800000u | ((wb >> 1) & 0x007FFF00u)) + (-0.9999847412109375f)) *
                   0.024543692606170259f;  // 2 pi / 2^8
  const float d2 = dl * dl;
  const float cd = fmaf(d2, fmaf(d2, 1.0f / 24.0f, -0.5f), 1.0f);
  const float sd = dl * fmaf(d2, fmaf(d2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
  const float c = fmaf(t.x, cd, -t.y * sd);
  const float s = fmaf(t.y, cd, t.x * sd);
  return make_float2(rho * c, rho * s);
}
GRF_DEV double2 box_muller_d(uint32_t wa, uint32_t wb) {
  const double ua = uniform_open_d(wa);
  const double ub = uniform_open_d(wb);
  const double rho = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  return make_double2(rho * c, rho * s);
}

// Algorithm 2 noise.  1-D: entry kd uses call kd >> 1, words 2 (kd & 1), 2 (kd & 1) + 1.
// 2-D / 3-D: with H = N1 / 2, entry (k1, kmid, kd) uses call
// ((k1 mod H) Nmid + kmid)(M + 1) + kd, words 2 [k1 >= H], 2 [k1 >= H] + 1
// (rows k1 and k1 + H share a call).
GRF_DEV uint64_t alg2_call_index(int k1, int kmid, int kd, int N1, int Nmid, int M) {
  const int H = N1 >> 1;
  const int r = k1 >= H ? k1 - H : k1;
  return ((uint64_t)r * (uint64_t)Nmid + (uint64_t)kmid) * (uint64_t)(M + 1) + (uint64_t)kd;
}
GRF_DEV float2 alg2_normals_grid(int k1, int kmid, int kd, int N1, int Nmid, int M, uint64_t key,
                                 const float2* trig) {
  const u32x4 w = philox_call(alg2_call_index(k1, kmid, kd, N1, Nmid, M), 0u, key);
  return k1 >= (N1 >> 1) ? box_muller(w.z, w.w, trig) : box_muller(w.x, w.y, trig);
}
GRF_DEV double2 alg2_normals_grid_d(int k1, int kmid, int kd, int N1, int Nmid, int M, uint64_t key) {
  const u32x4 w = philox_call(alg2_call_index(k1, kmid, kd, N1, Nmid, M), 0u, key);
  return k1 >= (N1 >> 1) ? box_muller_d(w.z, w.w) : box_muller_d(w.x, w.y);
}
GRF_DEV float2 alg2_normals_1d(int kd, uint64_t key, const float2* trig) {
  const u32x4 w = philox_call((uint64_t)(kd >> 1), 0u, key);
  return (kd & 1) ? box_muller(w.z, w.w, trig) : box_muller(w.x, w.y, trig);
}

// Hermitian noise xi_K of Algorithm 2 at a half-spectrum entry (k1, kmid, kd).
// Off the planes kd in {0, M}: (z_re + i z_im)/sqrt 2.  On the planes: the member
// of {K, -K} with the larger row-major index keeps its own normals, the other
// takes the conjugate; a self-conjugate K takes the real normal z_re.
GRF_DEV float2 alg2_xi_grid(int k1, int kmid, int kd, int N1, int Nmid, int M, uint64_t key,
                            const float2* trig) {
  const float r2 = 0.70710678118654752440f;
  if (kd != 0 && kd != M) {
    const float2 z = alg2_normals_grid(k1, kmid, kd, N1, Nmid, M, key, trig);
    return make_float2(z.x * r2, z.y * r2);
  }
  const int nk1 = k1 ? N1 - k1 : 0, nkm = kmid ? Nmid - kmid : 0;  // -K mod N for any even N
  const int row = k1 * Nmid + kmid, nrow = nk1 * Nmid + nkm;
  if (row == nrow) return make_float2(alg2_normals_grid(k1, kmid, kd, N1, Nmid, M, key, trig).x, 0.0f);
  if (row > nrow) {
    const float2 z = alg2_normals_grid(k1, kmid, kd, N1, Nmid, M, key, trig);
    return make_float2(z.x * r2, z.y * r2);
  }
  const float2 z = alg2_normals_grid(nk1, nkm, kd, N1, Nmid, M, key, trig);
  return make_float2(z.x * r2, -z.y * r2);
}
GRF_DEV double2 alg2_xi_grid_d(int k1, int kmid, int kd, int N1, int Nmid, int M, uint64_t key) {
  const double r2 = 0.70710678118654752440;
  if (kd != 0 && kd != M) {
    const double2 z = alg2_normals_grid_d(k1, kmid, kd, N1, Nmid, M, key);
    return make_double2(z.x * r2, z.y * r2);
  }
  // -K mod N for any even N (the FP64 form also takes sizes that are not powers of two)
  const int nk1 = k1 ? N1 - k1 : 0, nkm = kmid ? Nmid - kmid : 0;
  const int row = k1 * Nmid + kmid, nrow = nk1 * Nmid + nkm;
  if (row == nrow) return make_double2(alg2_normals_grid_d(k1, kmid, kd, N1, Nmid, M, key).x, 0.0);
  if (row > nrow) {
    const double2 z = alg2_normals_grid_d(k1, kmid, kd, N1, Nmid, M, key);
    return make_double2(z.x * r2, z.y * r2);
  }
  const double2 z = alg2_normals_grid_d(nk1, nkm, kd, N1, Nmid, M, key);
  return make_double2(z.x * r2, -z.y * r2);
}
// 1-D: the self-conjugate points are kd = 0 and kd = M; everything else is generic.
GRF_DEV float2 alg2_xi_1d(int kd, int M, uint64_t key, const float2* trig) {
  const float2 z = alg2_normals_1d(kd, key, trig);
  if (kd == 0 || kd == M) return make_float2(z.x, 0.0f);
  const float r2 = 0.70710678118654752440f;
  return make_float2(z.x * r2, z.y * r2);
}
GRF_DEV double2 alg2_xi_1d_d(int kd, int M, uint64_t key) {
  const u32x4 w = philox_call((uint64_t)(kd >> 1), 0u, key);
  const double2 z = (kd & 1) ? box_muller_d(w.z, w.w) : box_muller_d(w.x, w.y);
  if (kd == 0 || kd == M) return make_double2(z.x, 0.0);
  const double r2 = 0.70710678118654752440;
  return make_double2(z.x * r2, z.y * r2);
}

// Real normal of Algorithm 1 at flat grid index j: call j >> 2, pair t = (j & 3) >> 1,
// even j the cosine normal, odd j the sine normal.
GRF_DEV float alg1_normal(uint64_t j, uint64_t key, const float2* trig) {
  const u32x4 w = philox_call(j >> 2, 1u, key);
  const float2 z = ((j & 3) >> 1) ? box_muller(w.z, w.w, trig) : box_muller(w.x, w.y, trig);
  return (j & 1) ? z.y : z.x;
}
// Both reals of the pair (j even, j + 1) in one call.
GRF_DEV float2 alg1_normal_pair(uint64_t j_even, uint64_t key, const float2* trig) {
  const u32x4 w = philox_call(j_even >> 2, 1u, key);
  return ((j_even & 3) >> 1) ? box_muller(w.z, w.w, trig) : box_muller(w.x, w.y, trig);
}
GRF_DEV double alg1_normal_d(uint64_t j, uint64_t key) {
  const u32x4 w = philox_call(j >> 2, 1u, key);
  const double2 z = ((j & 3) >> 1) ? box_muller_d(w.z, w.w) : box_muller_d(w.x, w.y);
  return (j & 1) ? z.y : z.x;
}

}  // namespace grf
