// The noise + axis-1 pass of 2-D plans in pair mode (the pass that also forms
// the c2r split Z), specialised for the 256-thread radix-16 geometries:
// transform length N = 2^LN (256..4096), CC = 4096 / N column pairs per CTA,
// workspace tile T = TT.  Same arithmetic and same outputs as col_body_pair
// with SRC = COL_NOISE, MODE = COL_INV (bit for bit up to the
// rounding of the Box-Muller scale, see box_muller_half), with fewer
// instructions per entry:
//   - the field's Philox key is formed from the block index (uniform across
//     the CTA), so its round keys live in uniform registers;
//   - the 256 coarse Box-Muller angles are read from shared memory;
//   - Box-Muller returns the normals times 1/sqrt 2 directly (rho^2 = -ln u
//     instead of -2 ln u), the factor interior columns need (Lemma 1);
//   - the folded s_K index needs no min(): entries q < P/2 of a thread sit
//     below N/2 and the others above;
//   - store offsets are 32-bit within a field, with a compile-time tile, so
//     consecutive entries of a thread differ by one constant stride.
#pragma once
#include "bodies.cuh"

namespace grf {

// (rho / sqrt 2)(cos 2 pi u_b, sin 2 pi u_b) with rho = sqrt(-2 ln u_a): the
// same steps as box_muller, with -ln u_a in place of -2 ln u_a under the
// root and the coarse angles read from the shared-memory copy `strig`.
GRF_DEV float2 box_muller_half(uint32_t wa, uint32_t wb, const float2* strig) {
  const float ua = uniform_open(wa);
  const float ta = 1.0f - ua;
  const float near1 = ta * fmaf(ta, fmaf(ta, fmaf(ta, 0.25f, 0.333333343f), 0.5f), 1.0f);
  const float h = ta < 0.0078125f ? near1 : -__logf(ua);  // -ln u_a
  const float rho = h * rsqrtf(h);                          // sqrt(-ln u_a) = rho / sqrt 2
  const float2 t = strig[wb >> 24];
  const float dl = (__int_as_float(0x3F800000u | ((wb >> 1) & 0x007FFF00u)) + (-0.9999847412109375f)) *
                   0.024543692606170259f;
  const float d2 = dl * dl;
  const float cd = fmaf(d2, fmaf(d2, 1.0f / 24.0f, -0.5f), 1.0f);
  const float sd = dl * fmaf(d2, fmaf(d2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
  const float c = fmaf(t.x, cd, -t.y * sd);
  const float s = fmaf(t.y, cd, t.x * sd);
  return make_float2(rho * c, rho * s);
}

// Interior-column normals (z_re + i z_im) / sqrt 2 of the entries
// k1 = tau + TPT q of column (kmid, kd) (call ((k1 mod N1/2) Nmid + kmid)(M + 1)
// + kd, words 2 [k1 >= N1/2], +1): the rows k1 and k1 + N1/2 of a call are this
// thread's entries q and q + P/2.
template <int P, int TPT>
GRF_DEV void normals_half(float2 (&v)[P], int tau, int kmid, int kd, int Nmid, int M, uint64_t key,
                          const float2* strig) {
  const uint64_t stride = (uint64_t)TPT * (uint64_t)Nmid * (uint64_t)(M + 1);
  uint64_t call = ((uint64_t)tau * (uint64_t)Nmid + (uint64_t)kmid) * (uint64_t)(M + 1) + (uint64_t)kd;
#pragma unroll
  for (int i = 0; i < P / 2; ++i, call += stride) {
    const u32x4 w = philox_call(call, 0u, key);
    v[i] = box_muller_half(w.x, w.y, strig);
    v[i + P / 2] = box_muller_half(w.z, w.w, strig);
  }
}

// Shared memory: the transform's exchange buffer, the stash of column p's X
// (one slot per thread and entry) and the 256 coarse angles.
__host__ __device__ constexpr size_t noise_fast_smem_bytes(int N, int C) {
  return ((size_t)(N + N / 16) * C + (size_t)C * N + 256) * sizeof(float2);
}

template <int LN, int CC, int TT>
__global__ void __launch_bounds__(256, 3) noise_pair_fast(ColArgs a) {
  constexpr int P = 16, N = 1 << LN, TPT = N / P, NTHR = CC * TPT;
  static_assert(NTHR == 256, "256-thread geometries only");
  static_assert(TPT % TT == 0, "the tile must divide the thread stride");
  extern __shared__ float2 sm[];
  float2* stash = sm + (size_t)(N + N / 16) * CC;
  float2* strig = stash + (size_t)CC * N;
  const HalfGeom& g = a.g;
  strig[CtaCoordsHW{}.tid()] = __ldg(g.trig + CtaCoordsHW{}.tid());
  __syncthreads();

  const int M = g.M;
  const uint64_t key = field_key(g, blockIdx.z);  // uniform
  const float* stab = field_stab(g, blockIdx.z);
  float2 v[P];

  // One column kd of the pair: noise, s_K, the inverse FFT along axis 1; the
  // planes kd in {0, M} take the conjugation rule, invalid slots zeros.
  auto column = [&](int kd, bool valid) {
    const int t = CtaCoordsHW{}.tid();
    const int c = t & (CC - 1), tau = t / CC;
    const float* srow = stab + (size_t)kd * (N / 2 + 1);
    if (kd != 0 && kd != M) {
      normals_half<P, TPT>(v, tau, 0, kd, 1, M, key, strig);
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const float s = __ldg(srow + (q < P / 2 ? tau + TPT * q : N - tau - TPT * q));
        v[q] = cscale(v[q], s);
      }
    } else {
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const float s = __ldg(srow + (q < P / 2 ? tau + TPT * q : N - tau - TPT * q));
        v[q] = cscale(plane_xi(tau + TPT * q, 0, kd, N, 1, M, key, g.trig), s);
      }
    }
    if (!valid) {
#pragma unroll
      for (int q = 0; q < P; ++q) v[q] = make_float2(0.f, 0.f);
    }
    fft_core<P, +1>(v, sm, tau, c, CC, N, LN, a.tw, a.tws, NTHR);
  };

  {
    const int c = CtaCoordsHW{}.tid() & (CC - 1);
    const int p = (int)blockIdx.x * CC + c;
    column(p <= M / 2 ? p : 0, p <= M / 2);
  }
#pragma unroll
  for (int q = 0; q < P; ++q) stash[q * NTHR + CtaCoordsHW{}.tid()] = v[q];
  {
    const int c = CtaCoordsHW{}.tid() & (CC - 1);
    const int p = (int)blockIdx.x * CC + c;
    // pair M/2 is one column: its second transform only keeps the barriers in step
    column(p <= M / 2 ? M - p : 0, p <= M / 2 && p != M - p);
  }

  const int t = CtaCoordsHW{}.tid();
  const int c = t & (CC - 1), tau = t / CC;
  const int p = (int)blockIdx.x * CC + c;
  if (p > M / 2) return;
  const int ca = p, cb = M - p;
  const int ncols = M + 1;
  float2* out = a.out + (int64_t)blockIdx.z * a.bstride;
  // offset of (pos = tau + TPT q, col) in [pos / TT][col][pos % TT]
  const int base = (tau / TT) * (ncols * TT) + (tau & (TT - 1));
  const int qstride = TPT * ncols;
  const float2 w = __ldg(a.twz + p);
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const float2 xa = stash[q * NTHR + t];
    const float2 xb = ca == cb ? xa : v[q];
    const float2 A = make_float2(xa.x + xb.x, xa.y - xb.y);
    const float2 B = make_float2(xa.x - xb.x, xa.y + xb.y);
    const float2 wB = cmul(w, B);
    const int o = base + q * qstride;
    out[o + ca * TT] = make_float2(A.x - wB.y, A.y + wB.x);
    if (p != 0 && ca != cb) out[o + cb * TT] = make_float2(A.x + wB.y, wB.x - A.y);
  }
}

}  // namespace grf
