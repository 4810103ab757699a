// Plain FP64 form of the method: one field per launch sequence, nothing fused.
//   noise kernel (xi on the full grid, Hermitian by Eq. conj, or real z for
//   Algorithm 1) -> HBM; scale kernel (s_K, or s_K / sqrt(N_tot) after the
//   forward transform of Algorithm 1); radix-2 Stockham FFT, one launch per
//   stage, along every axis over the full complex grid; real part.
// It is the FP64 comparator of the fused FP32 path and the GRF_FP64 plans.
#include "kernels.h"
#include "common.cuh"
#include "plain64.h"

namespace grf {

struct Full64 {
  int d;
  int n[3];       // N_1..N_d (unused axes = 1)
  int M;          // N_d / 2
  uint32_t Q;
  int Nmid;       // N_2 for d = 3, else 1
  int N1;         // N_1 for d >= 2, else 1
};

// Full-grid flat index -> (k1, kmid, kd) in the d = 1/2/3 convention of H.
__device__ void split_full(int64_t idx, const Full64& f, int* k1, int* km, int* kd) {
  const int Nd = f.n[f.d - 1];
  *kd = (int)(idx % Nd);
  const int64_t r = idx / Nd;
  if (f.d == 3) {
    *km = (int)(r % f.n[1]);
    *k1 = (int)(r / f.n[1]);
  } else if (f.d == 2) {
    *km = 0;
    *k1 = (int)r;
  } else {
    *km = 0;
    *k1 = 0;
  }
}

__global__ void noise_full_alg2(double2* x, Full64 f, uint64_t key, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int k1, km, kd;
  split_full(i, f, &k1, &km, &kd);
  bool conj_it = false;
  if (kd > f.M) {  // outside H: xi_K = conj xi_{-K}
    kd = f.n[f.d - 1] - kd;
    k1 = k1 ? f.N1 - k1 : 0;
    km = km ? f.Nmid - km : 0;
    conj_it = true;
  }
  double2 xi = f.d == 1 ? alg2_xi_1d_d(kd, f.M, key) : alg2_xi_grid_d(k1, km, kd, f.N1, f.Nmid, f.M, key);
  if (conj_it) xi.y = -xi.y;
  x[i] = xi;
}

__global__ void noise_full_alg1(double2* x, uint64_t key, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  x[i] = make_double2(alg1_normal_d((uint64_t)i, key), 0.0);
}

// x_K *= factor * s_K, s from the FP64 folded table.
__global__ void scale_full(double2* x, const double* stab, Full64 f, double factor, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int k1, km, kd;
  split_full(i, f, &k1, &km, &kd);
  const int f1 = min(k1, f.N1 - k1), fm = min(km, f.Nmid - km), fd = min(kd, f.n[f.d - 1] - kd);
  const double s = stab[((int64_t)fd * (f.Nmid / 2 + 1) + fm) * (f.N1 / 2 + 1) + f1];
  x[i] = cscale(x[i], s * factor);
}

// One radix-2 Stockham stage along an axis of length n viewed as [outer][n][inner]:
// butterfly j < n/2 reads j, j + n/2 and writes (j / Ns) 2 Ns + j % Ns (+ Ns).
__global__ void stockham2_stage(const double2* __restrict__ x, double2* __restrict__ y, int n, int64_t inner,
                                int Ns, int dir, const double2* __restrict__ tw, int64_t total) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int64_t in = t % inner;
  const int64_t r = t / inner;
  const int half = n >> 1;
  const int j = (int)(r % half);
  const int64_t o = r / half;
  const int64_t base = o * n * inner + in;
  const double2 a = x[base + (int64_t)j * inner];
  const double2 b = x[base + (int64_t)(j + half) * inner];
  const int m = j & (Ns - 1);
  double2 w = tw[2 * Ns + m];  // exp(2 pi i m / (2 Ns))
  if (dir < 0) w.y = -w.y;
  const double2 wb = cmul(w, b);
  const int64_t od = (int64_t)((j - m) * 2 + m);
  y[base + od * inner] = cadd(a, wb);
  y[base + (od + Ns) * inner] = csub(a, wb);
}

// One Stockham stage of radix R (2 < R <= 7, odd) along an axis of length n
// (any n divisible by R): butterfly j < n/R reads j + q n/R (q < R), twists
// input q by exp(dir 2 pi i m q / (R Ns)) with m = j mod Ns, takes the R-point
// DFT and writes output q' to (j / Ns) R Ns + m + q' Ns.  After stages whose
// radices multiply to n the result is in natural order.  Twiddles come from
// sincospi of an exactly reduced fraction, in FP64.
__global__ void stockham_odd_stage(const double2* __restrict__ x, double2* __restrict__ y, int n, int64_t inner,
                                   int Ns, int R, int dir, int64_t total) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int64_t in = t % inner;
  const int64_t r = t / inner;
  const int nR = n / R;
  const int j = (int)(r % nR);
  const int64_t o = r / nR;
  const int64_t base = o * n * inner + in;
  const int m = j % Ns;
  const int64_t span = (int64_t)R * Ns;
  double2 v[7];
  for (int q = 0; q < R; ++q) {
    double2 a = x[base + (int64_t)(j + q * nR) * inner];
    if (q > 0 && m > 0) {
      double sn, cs;
      sincospi((double)((2 * (int64_t)m * q) % (2 * span)) / (double)span, &sn, &cs);
      a = cmul(a, make_double2(cs, dir > 0 ? sn : -sn));
    }
    v[q] = a;
  }
  double2 root[7];  // exp(dir 2 pi i h / R), h < R
  for (int h = 0; h < R; ++h) {
    double sn, cs;
    sincospi((double)(2 * h) / (double)R, &sn, &cs);
    root[h] = make_double2(cs, dir > 0 ? sn : -sn);
  }
  const int64_t od = (int64_t)(j - m) * R + m;
  for (int q2 = 0; q2 < R; ++q2) {
    double2 acc = v[0];
    for (int q = 1; q < R; ++q) acc = cadd(acc, cmul(v[q], root[(q * q2) % R]));
    y[base + (od + (int64_t)q2 * Ns) * inner] = acc;
  }
}

__global__ void real_part(const double2* x, double* out, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  out[i] = x[i].x;
}

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Full complex DFT along every axis; result ends in *cur (ping-pong with *other).
static cudaError_t fft_all_axes(double2** cur, double2** other, const Plain64Geom& g, int dir,
                                const double2* tw, cudaStream_t s) {
  int64_t outer = 1;
  for (int ax = 0; ax < g.d; ++ax) {
    const int n = g.n[ax];
    int64_t inner = 1;
    for (int b = ax + 1; b < g.d; ++b) inner *= g.n[b];
    // radix-2 stages for the power-of-two factor (spans 1, 2, 4, ...: the
    // twiddle table holds them), then one stage per odd prime factor
    int pow2 = 1;
    while (n % (2 * pow2) == 0) pow2 *= 2;
    int Ns = 1;
    for (; Ns < pow2; Ns *= 2) {
      const int64_t total = outer * (n / 2) * inner;
      stockham2_stage<<<nblk(total, 256), 256, 0, s>>>(*cur, *other, n, inner, Ns, dir, tw, total);
      double2* t = *cur;
      *cur = *other;
      *other = t;
    }
    int rest = n / pow2;
    for (int R : {3, 5, 7}) {
      while (rest % R == 0) {
        const int64_t total = outer * (n / R) * inner;
        stockham_odd_stage<<<nblk(total, 256), 256, 0, s>>>(*cur, *other, n, inner, Ns, R, dir, total);
        double2* t = *cur;
        *cur = *other;
        *other = t;
        Ns *= R;
        rest /= R;
      }
    }
    if (rest != 1) return cudaErrorInvalidValue;  // plan creation admits 2^a 3^b 5^c 7^e only
    outer *= n;
  }
  return cudaGetLastError();
}

cudaError_t plain64_field(const Plain64Geom& g, int alg, uint64_t key, const double* stab, const double2* tw,
                          double2* bufA, double2* bufB, double* out, cudaStream_t s) {
  Full64 f{};
  f.d = g.d;
  for (int i = 0; i < 3; ++i) f.n[i] = i < g.d ? g.n[i] : 1;
  f.M = g.n[g.d - 1] / 2;
  f.Q = (uint32_t)(f.M / 2 + 1);
  f.N1 = g.d >= 2 ? g.n[0] : 1;
  f.Nmid = g.d == 3 ? g.n[1] : 1;
  int64_t total = 1;
  for (int i = 0; i < g.d; ++i) total *= g.n[i];
  double2* cur = bufA;
  double2* other = bufB;
  if (alg == 2) {
    noise_full_alg2<<<nblk(total, 256), 256, 0, s>>>(cur, f, key, total);
    scale_full<<<nblk(total, 256), 256, 0, s>>>(cur, stab, f, 1.0, total);
  } else {
    noise_full_alg1<<<nblk(total, 256), 256, 0, s>>>(cur, key, total);
    cudaError_t e = fft_all_axes(&cur, &other, g, -1, tw, s);
    if (e != cudaSuccess) return e;
    scale_full<<<nblk(total, 256), 256, 0, s>>>(cur, stab, f, 1.0 / sqrt((double)total), total);
  }
  cudaError_t e = fft_all_axes(&cur, &other, g, +1, tw, s);
  if (e != cudaSuccess) return e;
  real_part<<<nblk(total, 256), 256, 0, s>>>(cur, out, total);
  return cudaGetLastError();
}

}  // namespace grf
