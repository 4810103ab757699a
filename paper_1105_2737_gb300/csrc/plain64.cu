// Plain form of the method: one field per launch sequence, nothing fused.
//   noise kernel (xi on the full grid, Hermitian by Eq. conj, or real z for
//   Algorithm 1) -> HBM; scale kernel (s_K, or s_K / sqrt(N_tot) after the
//   forward transform of Algorithm 1); Stockham FFT (radix 2, then 3, 5, 7),
//   one launch per stage, along every axis over the full complex grid; real part.
// In FP64 it is the comparator of the fused FP32 path and the GRF_FP64 plans;
// in FP32 it serves FP32 plans on grids that are not powers of two (the fused
// kernels take powers of two), with the noise of the fused path.
#include <type_traits>
#include "kernels.h"
#include "common.cuh"
#include "plain64.h"

namespace grf {

template <class R>
struct cplx;
template <>
struct cplx<float> {
  using t = float2;
  static __device__ t make(double re, double im) { return make_float2((float)re, (float)im); }
};
template <>
struct cplx<double> {
  using t = double2;
  static __device__ t make(double re, double im) { return make_double2(re, im); }
};

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

template <class R>
__global__ void noise_full_alg2(typename cplx<R>::t* x, Full64 f, uint64_t key, int64_t total, const float2* trig) {
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
  typename cplx<R>::t xi;
  if constexpr (std::is_same<R, double>::value)
    xi = f.d == 1 ? alg2_xi_1d_d(kd, f.M, key) : alg2_xi_grid_d(k1, km, kd, f.N1, f.Nmid, f.M, key);
  else
    xi = f.d == 1 ? alg2_xi_1d(kd, f.M, key, trig) : alg2_xi_grid(k1, km, kd, f.N1, f.Nmid, f.M, key, trig);
  if (conj_it) xi.y = -xi.y;
  x[i] = xi;
}

template <class R>
__global__ void noise_full_alg1(typename cplx<R>::t* x, uint64_t key, int64_t total, const float2* trig) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  if constexpr (std::is_same<R, double>::value)
    x[i] = make_double2(alg1_normal_d((uint64_t)i, key), 0.0);
  else
    x[i] = make_float2(alg1_normal((uint64_t)i, key, trig), 0.0f);
}

// x_K *= factor * s_K, s from the folded table.
template <class R>
__global__ void scale_full(typename cplx<R>::t* x, const R* stab, Full64 f, R factor, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int k1, km, kd;
  split_full(i, f, &k1, &km, &kd);
  const int f1 = min(k1, f.N1 - k1), fm = min(km, f.Nmid - km), fd = min(kd, f.n[f.d - 1] - kd);
  const R s = stab[((int64_t)fd * (f.Nmid / 2 + 1) + fm) * (f.N1 / 2 + 1) + f1];
  x[i] = cscale(x[i], s * factor);
}

// One radix-2 Stockham stage along an axis of length n viewed as [outer][n][inner]:
// butterfly j < n/2 reads j, j + n/2 and writes (j / Ns) 2 Ns + j % Ns (+ Ns).
// IX: the index type, 32-bit when the grid has fewer than 2^31 points (the
// divisions below are then 32-bit), else 64-bit.
template <class R, class IX>
__global__ void stockham2_stage(const typename cplx<R>::t* __restrict__ x, typename cplx<R>::t* __restrict__ y, int n,
                                IX inner, int Ns, int dir, const typename cplx<R>::t* __restrict__ tw, IX total) {
  const IX t = (IX)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const IX in = t % inner;
  const IX r = t / inner;
  const int half = n >> 1;
  const int j = (int)(r % half);
  const IX o = r / half;
  const IX base = o * n * inner + in;
  const auto a = x[base + (IX)j * inner];
  const auto b = x[base + (IX)(j + half) * inner];
  const int m = j & (Ns - 1);
  auto w = tw[2 * Ns + m];  // exp(2 pi i m / (2 Ns))
  if (dir < 0) w.y = -w.y;
  const auto wb = cmul(w, b);
  const IX od = (IX)((j - m) * 2 + m);
  y[base + od * inner] = cadd(a, wb);
  y[base + (od + Ns) * inner] = csub(a, wb);
}

// One Stockham stage of radix R (2 < R <= 7, odd) along an axis of length n
// (any n divisible by R): butterfly j < n/R reads j + q n/R (q < R), twists
// input q by exp(dir 2 pi i m q / (R Ns)) with m = j mod Ns, takes the R-point
// DFT and writes output q' to (j / Ns) R Ns + m + q' Ns.  After stages whose
// radices multiply to n the result is in natural order.  Every twiddle is an
// entry of the axis table twn[k] = exp(2 pi i k / n) (R Ns divides n):
// exp(2 pi i m q / (R Ns)) = twn[m q n / (R Ns)] (m q < R Ns), and the DFT's
// roots exp(2 pi i h / R) = twn[h n / R].
template <class T, int R, class IX>
__global__ void stockham_odd_stage(const typename cplx<T>::t* __restrict__ x, typename cplx<T>::t* __restrict__ y,
                                   int n, IX inner, int Ns, int dir, const typename cplx<T>::t* __restrict__ twn,
                                   IX total) {
  using C = cplx<T>;
  const IX t = (IX)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const IX in = t % inner;
  const IX r = t / inner;
  const int nR = n / R;
  const int j = (int)(r % nR);
  const IX o = r / nR;
  const IX base = o * n * inner + in;
  const int m = j % Ns;
  const int step = n / (R * Ns);  // twn index of exp(2 pi i / (R Ns))
  typename C::t v[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    typename C::t a = x[base + (IX)(j + q * nR) * inner];
    if (q > 0 && m > 0) {
      typename C::t w = twn[m * q * step];
      if (dir < 0) w.y = -w.y;
      a = cmul(a, w);
    }
    v[q] = a;
  }
  typename C::t root[R];  // exp(dir 2 pi i h / R), h < R
#pragma unroll
  for (int h = 0; h < R; ++h) {
    root[h] = twn[h * nR];
    if (dir < 0) root[h].y = -root[h].y;
  }
  const IX od = (IX)(j - m) * R + m;
#pragma unroll
  for (int q2 = 0; q2 < R; ++q2) {
    typename C::t acc = v[0];
#pragma unroll
    for (int q = 1; q < R; ++q) acc = cadd(acc, cmul(v[q], root[(q * q2) % R]));
    y[base + (od + (IX)q2 * Ns) * inner] = acc;
  }
}

template <class T, class IX>
static void launch_odd_stage(int R, const typename cplx<T>::t* x, typename cplx<T>::t* y, int n, IX inner, int Ns,
                             int dir, const typename cplx<T>::t* twn, IX total, cudaStream_t s) {
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (R == 3) stockham_odd_stage<T, 3, IX><<<blocks, 256, 0, s>>>(x, y, n, inner, Ns, dir, twn, total);
  else if (R == 5) stockham_odd_stage<T, 5, IX><<<blocks, 256, 0, s>>>(x, y, n, inner, Ns, dir, twn, total);
  else stockham_odd_stage<T, 7, IX><<<blocks, 256, 0, s>>>(x, y, n, inner, Ns, dir, twn, total);
}

template <class R>
__global__ void real_part(const typename cplx<R>::t* x, R* out, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  out[i] = x[i].x;
}

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Full complex DFT along every axis; result ends in *cur (ping-pong with *other).
template <class R>
static cudaError_t fft_all_axes(typename cplx<R>::t** cur, typename cplx<R>::t** other, const Plain64Geom& g, int dir,
                                const typename cplx<R>::t* tw, const typename cplx<R>::t* const* twax, cudaStream_t s) {
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
    const bool small = outer * n * inner < ((int64_t)1 << 31);  // 32-bit indices
    for (; Ns < pow2; Ns *= 2) {
      const int64_t total = outer * (n / 2) * inner;
      if (small)
        stockham2_stage<R, int><<<nblk(total, 256), 256, 0, s>>>(*cur, *other, n, (int)inner, Ns, dir, tw, (int)total);
      else
        stockham2_stage<R, int64_t><<<nblk(total, 256), 256, 0, s>>>(*cur, *other, n, inner, Ns, dir, tw, total);
      auto t = *cur;
      *cur = *other;
      *other = t;
    }
    int rest = n / pow2;
    for (int Rd : {3, 5, 7}) {
      while (rest % Rd == 0) {
        const int64_t total = outer * (n / Rd) * inner;
        if (!twax || !twax[ax]) return cudaErrorInvalidValue;
        if (small)
          launch_odd_stage<R, int>(Rd, *cur, *other, n, (int)inner, Ns, dir, twax[ax], (int)total, s);
        else
          launch_odd_stage<R, int64_t>(Rd, *cur, *other, n, inner, Ns, dir, twax[ax], total, s);
        auto t = *cur;
        *cur = *other;
        *other = t;
        Ns *= Rd;
        rest /= Rd;
      }
    }
    if (rest != 1) return cudaErrorInvalidValue;  // plan creation admits 2^a 3^b 5^c 7^e only
    outer *= n;
  }
  return cudaGetLastError();
}

template <class R>
static cudaError_t plain_field(const Plain64Geom& g, int alg, uint64_t key, const R* stab,
                               const typename cplx<R>::t* tw, const typename cplx<R>::t* const* twax,
                               const float2* trig, typename cplx<R>::t* bufA, typename cplx<R>::t* bufB, R* out,
                               cudaStream_t s) {
  Full64 f{};
  f.d = g.d;
  for (int i = 0; i < 3; ++i) f.n[i] = i < g.d ? g.n[i] : 1;
  f.M = g.n[g.d - 1] / 2;
  f.Q = (uint32_t)(f.M / 2 + 1);
  f.N1 = g.d >= 2 ? g.n[0] : 1;
  f.Nmid = g.d == 3 ? g.n[1] : 1;
  int64_t total = 1;
  for (int i = 0; i < g.d; ++i) total *= g.n[i];
  auto cur = bufA;
  auto other = bufB;
  if (alg == 2) {
    noise_full_alg2<R><<<nblk(total, 256), 256, 0, s>>>(cur, f, key, total, trig);
    scale_full<R><<<nblk(total, 256), 256, 0, s>>>(cur, stab, f, (R)1, total);
  } else {
    noise_full_alg1<R><<<nblk(total, 256), 256, 0, s>>>(cur, key, total, trig);
    cudaError_t e = fft_all_axes<R>(&cur, &other, g, -1, tw, twax, s);
    if (e != cudaSuccess) return e;
    scale_full<R><<<nblk(total, 256), 256, 0, s>>>(cur, stab, f, (R)(1.0 / sqrt((double)total)), total);
  }
  cudaError_t e = fft_all_axes<R>(&cur, &other, g, +1, tw, twax, s);
  if (e != cudaSuccess) return e;
  real_part<R><<<nblk(total, 256), 256, 0, s>>>(cur, out, total);
  return cudaGetLastError();
}

cudaError_t plain64_field(const Plain64Geom& g, int alg, uint64_t key, const double* stab, const double2* tw,
                          const double2* const* twax, double2* bufA, double2* bufB, double* out, cudaStream_t s) {
  return plain_field<double>(g, alg, key, stab, tw, twax, nullptr, bufA, bufB, out, s);
}

cudaError_t plain32_field(const Plain64Geom& g, int alg, uint64_t key, const float* stab, const float2* tw,
                          const float2* const* twax, const float2* trig, float2* bufA, float2* bufB, float* out,
                          cudaStream_t s) {
  return plain_field<float>(g, alg, key, stab, tw, twax, trig, bufA, bufB, out, s);
}

// twn[k] = exp(2 pi i k / n), k < n, from sincospi of the exact fraction 2k/n in FP64.
template <class R>
__global__ void axis_twiddle_kernel(typename cplx<R>::t* twn, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double sn, cs;
  sincospi(2.0 * (double)k / (double)n, &sn, &cs);
  twn[k] = cplx<R>::make(cs, sn);
}

cudaError_t build_axis_twiddles(double2* twn, int n, cudaStream_t s) {
  axis_twiddle_kernel<double><<<nblk(n, 256), 256, 0, s>>>(twn, n);
  return cudaGetLastError();
}
cudaError_t build_axis_twiddles(float2* twn, int n, cudaStream_t s) {
  axis_twiddle_kernel<float><<<nblk(n, 256), 256, 0, s>>>(twn, n);
  return cudaGetLastError();
}

}  // namespace grf
