// Plan-time tables, computed in FP64 on the device and rounded to FP32:
//  * twiddles exp(2 pi i k / L) for every power of two L up to a maximum,
//    stored at tw[L + k] (k < L);
//  * s_K = sqrt(S(p_K) / |D|) on the folded half spectrum, stored
//    (N_d/2+1) x (N_2/2+1) x (N_1/2+1) with axis 1 fastest (S depends on |p_i| only; §2 rules a), e),
//    Eq. drf), and for the adjoint d s_K / d ell and d s_K / d nu.
#include "kernels.h"
#include "common.cuh"
#include <math.h>

namespace grf {

__global__ void twiddle_kernel(float2* tw, int total) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  if (i == 0) {
    tw[0] = make_float2(1.f, 0.f);
    return;
  }
  const int L = 1 << (31 - __clz(i));
  const int k = i - L;
  double s, c;
  sincospi(2.0 * (double)k / (double)L, &s, &c);
  tw[i] = make_float2((float)c, (float)s);
}

__global__ void twiddle_kernel_d(double2* tw, int total) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  if (i == 0) {
    tw[0] = make_double2(1.0, 0.0);
    return;
  }
  const int L = 1 << (31 - __clz(i));
  const int k = i - L;
  double s, c;
  sincospi(2.0 * (double)k / (double)L, &s, &c);
  tw[i] = make_double2(c, s);
}

// Stage tables, per radix R in (16, 8, 4) and span Ns in (R, R^2, ...):
// entry (r - 1) Ns + m = exp(2 pi i m r / (R Ns)), r = 1..R-1, m < Ns.
__global__ void stage_table_kernel(float2* tws) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kStageTableEntries) return;
  double sn, cs;
  if (i >= kStageTableMain) {  // final small stages: span 16 (176 entries), then 256
    const int Ns = i < kStageTableMain + 11 * 16 ? 16 : 256;
    const int loc = i - (Ns == 16 ? kStageTableMain : kStageTableMain + 11 * 16);
    const int R = loc < Ns ? 2 : (loc < 4 * Ns ? 4 : 8);
    const int e = loc - (R == 2 ? 0 : (R == 4 ? Ns : 4 * Ns));
    const int r = e / Ns + 1, j = e % Ns;
    sincospi(2.0 * (double)(j * r) / (double)(R * Ns), &sn, &cs);
    tws[i] = make_float2((float)cs, (float)sn);
    return;
  }
  const int R = i < 4080 ? 16 : (i < 8168 ? 8 : 4);
  int loc = i < 4080 ? i : (i < 8168 ? i - 4080 : i - 8168);
  int Ns = R;
  while (loc >= (R - 1) * Ns) {
    loc -= (R - 1) * Ns;
    Ns *= R;
  }
  const int r = loc / Ns + 1, m = loc % Ns;
  sincospi(2.0 * (double)((int64_t)m * r) / (double)(R * Ns), &sn, &cs);
  tws[i] = make_float2((float)cs, (float)sn);
}

cudaError_t build_twiddles(float2* tw, int maxlen, cudaStream_t s) {
  const int total = 2 * maxlen;
  twiddle_kernel<<<(total + 255) / 256, 256, 0, s>>>(tw, total);
  stage_table_kernel<<<(kStageTableEntries + 255) / 256, 256, 0, s>>>(tw + total);
  return cudaGetLastError();
}

__global__ void stab_fourstep_kernel(float* stabT, const float* stab, int A, int B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)A * B) return;
  const int k1 = (int)(i / B), k2 = (int)(i - (int64_t)k1 * B);
  stabT[i] = stab[k1 + (int64_t)A * k2];
}

cudaError_t build_stab_fourstep(float* stabT, const float* stab, int A, int B, cudaStream_t s) {
  const int64_t n = (int64_t)A * B;
  stab_fourstep_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(stabT, stab, A, B);
  return cudaGetLastError();
}

cudaError_t build_twiddles_d(double2* tw, int maxlen, cudaStream_t s) {
  const int total = 2 * maxlen;
  twiddle_kernel_d<<<(total + 255) / 256, 256, 0, s>>>(tw, total);
  return cudaGetLastError();
}

struct DevSpec {
  int family, d;
  double coef;  // sigma^2 c / |D| * scale (Matern), analogues for the others
  double ell, nu, m;
  int k, l, n;
  double invL[3];
  int F[3];            // folded extents per axis of the table (1 for absent axes)
  int axis_of[3];      // table dimension t -> physical axis index (or -1)
  double dig;          // psi(nu + d/2) - psi(nu)
  double sigma;
};

// S(p)/|D| * scale and its log-derivatives at one folded entry.  The table is
// stored [kd][fmid][f1] (axis 1 fastest): the column kernels, whose lanes run
// along axis 1, then read consecutive entries.
__device__ void spectral_entry(const DevSpec& sp, int64_t idx, double* S, double* dl, double* dn) {
  const int i0 = (int)(idx % sp.F[0]);
  const int64_t r = idx / sp.F[0];
  const int i1 = (int)(r % sp.F[1]);
  const int i2 = (int)(r / sp.F[1]);
  const int f[3] = {i0, i1, i2};
  double p[3] = {0, 0, 0};
  double p2 = 0.0;
  for (int t = 0; t < 3; ++t) {
    if (sp.axis_of[t] >= 0) {
      p[t] = (double)f[t] * sp.invL[sp.axis_of[t]];
      p2 += p[t] * p[t];
    }
  }
  const double PI = 3.141592653589793238462643383279502884;
  const int d = sp.d;
  if (sp.family == 0) {  // Matern
    const double w2 = 4.0 * PI * PI * p2;
    const double a = sp.nu + 0.5 * d;
    const double den = 1.0 + sp.ell * sp.ell * w2;
    *S = sp.coef * pow(den, -a);
    *dl = d / sp.ell - a * 2.0 * sp.ell * w2 / den;
    *dn = sp.dig - log(den);
  } else if (sp.family == 1) {  // Gaussian
    *S = sp.coef * exp(-2.0 * PI * PI * sp.ell * sp.ell * p2);
    *dl = d / sp.ell - 4.0 * PI * PI * sp.ell * p2;
    *dn = 0.0;
  } else {  // paper polynomial family (§4)
    double s2k = 0.0;
    for (int t = 0; t < 3; ++t)
      if (sp.axis_of[t] >= 0) s2k += pow(p[t], 2.0 * sp.k);
    *S = sp.coef * pow(pow(sp.m, (double)(sp.k * sp.l)) + pow(s2k, (double)sp.l), -(double)sp.n);
    *dl = 0.0;
    *dn = 0.0;
  }
}

__global__ void stab_kernel(float* stab, float* dstab, DevSpec sp, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  double S, dl, dn;
  spectral_entry(sp, i, &S, &dl, &dn);
  const double s = sqrt(S);
  stab[i] = (float)s;
  if (dstab) {
    dstab[i] = (float)(0.5 * s * dl);
    dstab[total + i] = (float)(0.5 * s * dn);
  }
}

__global__ void stab_kernel_d(double* stab, DevSpec sp, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  double S, dl, dn;
  spectral_entry(sp, i, &S, &dl, &dn);
  stab[i] = sqrt(S);
}

static DevSpec make_devspec(const SpecParams& sp, double dig) {
  DevSpec d{};
  d.family = sp.family;
  d.d = sp.d;
  d.ell = sp.ell;
  d.nu = sp.nu;
  d.m = sp.m;
  d.k = sp.k;
  d.l = sp.l;
  d.n = sp.n;
  d.dig = dig;
  d.sigma = sp.sigma;
  double vol = 1.0;
  for (int i = 0; i < sp.d; ++i) {
    vol *= sp.L[i];
    d.invL[i] = 1.0 / sp.L[i];
  }
  const double PI = 3.141592653589793238462643383279502884;
  if (sp.family == 0) {
    const double c = pow(2.0 * sqrt(PI) * sp.ell, sp.d) * exp(lgamma(sp.nu + 0.5 * sp.d) - lgamma(sp.nu));
    d.coef = sp.sigma * sp.sigma * c / vol * sp.scale;
  } else if (sp.family == 1) {
    d.coef = sp.sigma * sp.sigma * pow(2.0 * PI * sp.ell * sp.ell, 0.5 * sp.d) / vol * sp.scale;
  } else {
    d.coef = sp.sigma * sp.sigma / vol * sp.scale;
  }
  // table dims: t = 0 <-> axis 1 (if d >= 2), t = 1 <-> axis 2 (if d == 3), t = 2 <-> axis d
  for (int t = 0; t < 3; ++t) {
    d.F[t] = 1;
    d.axis_of[t] = -1;
  }
  d.F[2] = sp.nn[sp.d - 1] / 2 + 1;
  d.axis_of[2] = sp.d - 1;
  if (sp.d >= 2) {
    d.F[0] = sp.nn[0] / 2 + 1;
    d.axis_of[0] = 0;
  }
  if (sp.d == 3) {
    d.F[1] = sp.nn[1] / 2 + 1;
    d.axis_of[1] = 1;
  }
  return d;
}

cudaError_t build_stab(float* stab, float* dstab, const SpecParams& sp, double dig, cudaStream_t s) {
  const DevSpec d = make_devspec(sp, dig);
  const int64_t total = (int64_t)d.F[0] * d.F[1] * d.F[2];
  stab_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(stab, dstab, d, total);
  return cudaGetLastError();
}

cudaError_t build_stab_d(double* stab, const SpecParams& sp, cudaStream_t s) {
  const DevSpec d = make_devspec(sp, 0.0);
  const int64_t total = (int64_t)d.F[0] * d.F[1] * d.F[2];
  stab_kernel_d<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(stab, d, total);
  return cudaGetLastError();
}

// t_K of the boundary-condition fields: the folded-table machinery with the
// table dimensions mapped so that the last axis is fastest (field layout), the
// edges doubled (the mirrored box), and the per-axis factor of the extension.
__global__ void bc_table_kernel(float* tab, DevSpec sp, int bc, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  double S, dl, dn;
  spectral_entry(sp, i, &S, &dl, &dn);
  const int f[3] = {(int)(i % sp.F[0]), (int)((i / sp.F[0]) % sp.F[1]), (int)(i / ((int64_t)sp.F[0] * sp.F[1]))};
  double u = 1.0;
  for (int t = 0; t < 3; ++t) {
    if (sp.axis_of[t] < 0) continue;
    const bool edge = f[t] == 0 || f[t] == sp.F[t] - 1;
    u *= edge ? (bc == 1 ? 1.0 : 0.0) : 0.70710678118654752440;
  }
  tab[i] = (float)(sqrt(S) * u);
}

cudaError_t build_bc_table(float* tab, const SpecParams& sp, int bc, cudaStream_t s) {
  SpecParams s2 = sp;
  for (int i = 0; i < sp.d; ++i) s2.L[i] = 2.0 * sp.L[i];
  DevSpec d = make_devspec(s2, 0.0);
  // table dimension 0 (fastest) <-> the last axis, 1 <-> axis 2 of a 3-D
  // grid, 2 <-> axis 1; N_i + 1 entries each
  for (int t = 0; t < 3; ++t) {
    d.F[t] = 1;
    d.axis_of[t] = -1;
  }
  d.F[0] = sp.nn[sp.d - 1] + 1;
  d.axis_of[0] = sp.d - 1;
  if (sp.d == 3) {
    d.F[1] = sp.nn[1] + 1;
    d.axis_of[1] = 1;
  }
  if (sp.d >= 2) {
    d.F[2] = sp.nn[0] + 1;
    d.axis_of[2] = 0;
  }
  const int64_t total = (int64_t)d.F[0] * d.F[1] * d.F[2];
  bc_table_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(tab, d, bc, total);
  return cudaGetLastError();
}

// out[f * 3 + t] = sum_i partial[(f * nblk + i) * 3 + t], summed in index order.
__global__ void reduce_partials_kernel(const double* partial, int64_t nblk, int64_t nfields, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nfields * 3) return;
  const int64_t f = i / 3;
  const int t = (int)(i - f * 3);
  double acc = 0.0;
  for (int64_t b = 0; b < nblk; ++b) acc += partial[(f * nblk + b) * 3 + t];
  out[i] = acc;
}

cudaError_t reduce_partials(const double* partial, int64_t nblk, int64_t nfields, double* out, cudaStream_t s) {
  const int64_t n = nfields * 3;
  reduce_partials_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(partial, nblk, nfields, out);
  return cudaGetLastError();
}

__global__ void philox_words_kernel(uint64_t key, uint32_t tag, uint64_t q0, int64_t count, uint32_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const u32x4 w = philox_call(q0 + (uint64_t)i, tag, key);
  out[4 * i] = w.x;
  out[4 * i + 1] = w.y;
  out[4 * i + 2] = w.z;
  out[4 * i + 3] = w.w;
}

cudaError_t philox_words(uint64_t key, uint32_t tag, uint64_t q0, int64_t count, uint32_t* out, cudaStream_t s) {
  philox_words_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(key, tag, q0, count, out);
  return cudaGetLastError();
}

}  // namespace grf
