// CTA-level Stockham FFT engine (FP32 data, twiddles from FP64-built tables).
//
// A CTA transforms C independent sequences of length N = TPT * P at once; each
// thread owns P points of one sequence in registers.  Thread (c, tau) holds
// the points at positions tau + TPT * q, q = 0..P-1, both on entry (input
// order) and on exit (output order): the Stockham autosort formulation
// (stage with radix R and span Ns: butterfly j reads j + r N/R and writes
// (j / Ns) Ns R + j % Ns + r Ns) leaves the first stage's read set and the
// last stage's write set on the same registers.  Stages are radix 16 (an
// in-register DIF network) with one final radix 2/4/8 stage if log2 N is not
// a multiple of 4; between stages the points go through shared memory, in an
// interleaved layout (c fastest) padded by one element every 16 positions so
// that the stage writes of a half warp hit distinct banks.
#pragma once
#include <type_traits>
#include "common.cuh"
#include "kernels.h"

namespace grf {

template <int I, int E, class F>
GRF_DEV void static_for(F&& f) {
  if constexpr (I < E) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, E>(f);
  }
}

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }
__host__ __device__ constexpr int bitrevc(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r = (r << 1) | ((x >> i) & 1);
  return r;
}

// cos and sin of 2 pi e / 16.
constexpr double kC16[16] = {1.0,
                             0.92387953251128675613,
                             0.70710678118654752440,
                             0.38268343236508977173,
                             0.0,
                             -0.38268343236508977173,
                             -0.70710678118654752440,
                             -0.92387953251128675613,
                             -1.0,
                             -0.92387953251128675613,
                             -0.70710678118654752440,
                             -0.38268343236508977173,
                             0.0,
                             0.38268343236508977173,
                             0.70710678118654752440,
                             0.92387953251128675613};
constexpr double kS16[16] = {0.0,
                             0.38268343236508977173,
                             0.70710678118654752440,
                             0.92387953251128675613,
                             1.0,
                             0.92387953251128675613,
                             0.70710678118654752440,
                             0.38268343236508977173,
                             0.0,
                             -0.38268343236508977173,
                             -0.70710678118654752440,
                             -0.92387953251128675613,
                             -1.0,
                             -0.92387953251128675613,
                             -0.70710678118654752440,
                             -0.38268343236508977173};

// a * exp(DIR 2 pi i E / R), R <= 16, with the trivial factors written out.
template <int E, int R, int DIR>
GRF_DEV float2 twmul(float2 a) {
  constexpr int e = ((E * (16 / R)) % 16 + 16) % 16;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (e == 8) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (e == 4) {
    if constexpr (DIR > 0) return make_float2(-a.y, a.x);
    else return make_float2(a.y, -a.x);
  } else if constexpr (e == 12) {
    if constexpr (DIR > 0) return make_float2(a.y, -a.x);
    else return make_float2(-a.y, a.x);
  } else {
    constexpr float c = (float)kC16[e];
    constexpr float s = DIR > 0 ? (float)kS16[e] : -(float)kS16[e];
    return make_float2(fmaf(c, a.x, -s * a.y), fmaf(c, a.y, s * a.x));
  }
}

// In-register DFT of R points (R a power of two <= 16):
// X[k] = sum_n x[n] exp(DIR 2 pi i n k / R).  x[STRIDE * i + OFF] holds point i.
template <int R, int DIR, int STRIDE, int OFF, int NV>
GRF_DEV void dft_regs(float2 (&x)[NV]) {
  if constexpr (R == 1) {
    return;
  } else {
    constexpr int LG = ilog2c(R);
    static_for<0, LG>([&](auto lv) {
      constexpr int span = R >> (decltype(lv)::value + 1);
      static_for<0, R / (2 * span)>([&](auto blk) {
        static_for<0, span>([&](auto k) {
          constexpr int i0 = decltype(blk)::value * 2 * span + decltype(k)::value;
          constexpr int i1 = i0 + span;
          const float2 a = x[STRIDE * i0 + OFF], b = x[STRIDE * i1 + OFF];
          x[STRIDE * i0 + OFF] = cadd(a, b);
          x[STRIDE * i1 + OFF] = twmul<decltype(k)::value*(R / (2 * span)), R, DIR>(csub(a, b));
        });
      });
    });
    float2 y[R];
    static_for<0, R>([&](auto k) { y[decltype(k)::value] = x[STRIDE * bitrevc(decltype(k)::value, LG) + OFF]; });
    static_for<0, R>([&](auto k) { x[STRIDE * decltype(k)::value + OFF] = y[decltype(k)::value]; });
  }
}

// Barrier over the first `nthr` threads of the CTA (all of them in the regular
// kernels; a multiple of 32 when a persistent CTA runs a smaller work item).
GRF_DEV void cta_sync(int nthr) {
  if (nthr == (int)blockDim.x) {
    __syncthreads();
  } else {
    asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
  }
}

// Padded shared-memory position.
GRF_DEV int spad(int p) { return p + (p >> 4); }
__host__ __device__ inline int spad_h(int p) { return p + (p >> 4); }

GRF_DEV float2 tw_load(const float2* __restrict__ tw, int k, int dir) {
  const float2 w = __ldg(tw + k);
  return dir > 0 ? w : make_float2(w.x, -w.y);
}

// One final stage of radix R < P: each thread does P/R butterflies j = tau + u TPT
// on registers v[u + r P/R]; Ns = N/R so the twiddle is exp(DIR 2 pi i j r / N).
// With radix-16 stages before it (P = 16, Ns = 16 or 256) the twiddles come
// from the small-stage table, entry (r - 1) Ns + j (lanes with consecutive j
// read consecutive entries); otherwise from tw[j r].
template <int P, int R, int DIR>
GRF_DEV void last_small_stage(float2 (&v)[P], int tau, int TPT, const float2* __restrict__ tw,
                              const float2* __restrict__ tws) {
  constexpr int U = P / R;
  const int Ns = TPT * U;
  const bool table = P == 16 && (Ns == 16 || Ns == 256);
  const float2* st = tws + (Ns == 16 ? small_stage_offset(R, 16) : small_stage_offset(R, 256));
  static_for<0, U>([&](auto uu) {
    constexpr int u = decltype(uu)::value;
    const int j = tau + u * TPT;
    static_for<1, R>([&](auto rr) {
      constexpr int r = decltype(rr)::value;
      const float2 w = table ? tw_load(st, (r - 1) * Ns + j, DIR) : tw_load(tw, j * r, DIR);
      v[u + r * U] = cmul(v[u + r * U], w);
    });
    dft_regs<R, DIR, U, u>(v);
  });
}

// Offset of the radix-P stage tables inside `tws` (radix 16, then 8, then 4).
template <int P>
__host__ __device__ constexpr int stage_table_offset() {
  return P == 16 ? 0 : (P == 8 ? 4080 : 4080 + 4088);
}

// C sequences of length N (runtime power of two, N = TPT * P, N >= P) per CTA,
// radix P in {4, 8, 16} (P = N <= 2 is a single butterfly).
//   v   : this thread's points (positions tau + TPT q)
//   sm  : shared buffer of at least spad(N) * C float2 (unused if N == P)
//   tw  : tw[k] = exp(+2 pi i k / N), k < N (FP64-built, FP32-rounded)
//   tws : stage tables: for radix P and span Ns (P, P^2, ...) the entries
//         (r - 1) Ns + m = exp(+2 pi i m r / (P Ns)), r = 1..P-1, m < Ns, so
//         that the lanes of a warp (consecutive m) read consecutive entries
//   nthr: threads taking part (C * N / P), the barrier count of every exchange
// Every exchange starts with a barrier, so the caller may have used `sm` just
// before; after return other threads may still read `sm`.
// PF: load the next stage's twiddles before the exchange (latency hidden
// behind it, P - 1 more live float2); without, load them after it (fewer
// registers, for kernels held to 64 registers).
template <int P, int DIR, bool PF = true>
GRF_DEV void fft_core(float2 (&v)[P], float2* sm, int tau, int c, int C, int N, int logN,
                      const float2* __restrict__ tw, const float2* __restrict__ tws, int nthr) {
  if constexpr (P == 1) {
    return;
  } else if constexpr (P == 2) {
    dft_regs<2, DIR, 1, 0>(v);  // N == 2
  } else {
    constexpr int LP = ilog2c(P);
    if (N == P) {  // a single in-register stage
      dft_regs<P, DIR, 1, 0>(v);
      return;
    }
    const int TPT = N >> LP;
    const int nP = logN / LP;
    const int rl = logN - nP * LP;
    // read positions tau + TPT q: spad is linear in q when TPT is a multiple of 16
    const int rd0 = spad(tau) * C + c;
    const int rdq = (TPT + (TPT >> 4)) * C;
    const float2* tab = tws + stage_table_offset<P>();
    int Ns = 1;
    int off = 0;
    float2 w[PF ? P - 1 : 1];  // twiddles of the next stage, loaded one stage ahead
    for (int s = 0; s < nP; ++s) {
      const int m = tau & (Ns - 1);
      if constexpr (PF) {
        if (Ns > 1) {
#pragma unroll
          for (int r = 1; r < P; ++r) v[r] = cmul(v[r], make_float2(w[r - 1].x, DIR > 0 ? w[r - 1].y : -w[r - 1].y));
        }
        if (s + 1 < nP) {  // span of the next stage: P Ns
          const float2* t = tab + off + (tau & (P * Ns - 1));
#pragma unroll
          for (int r = 1; r < P; ++r) w[r - 1] = __ldg(t + (r - 1) * (P * Ns));
          off += (P - 1) * P * Ns;
        }
      } else if (Ns > 1) {  // this stage's table: span Ns, entries (r - 1) Ns + m
        const float2* t = tab + off + m;
#pragma unroll
        for (int r = 1; r < P; ++r) {
          const float2 ww = __ldg(t + (r - 1) * Ns);
          v[r] = cmul(v[r], make_float2(ww.x, DIR > 0 ? ww.y : -ww.y));
        }
        off += (P - 1) * Ns;
      }
      dft_regs<P, DIR, 1, 0>(v);
      const bool last = (s == nP - 1) && rl == 0;
      if (!last) {
        // write positions (j / Ns) Ns P + j % Ns + r Ns, j = tau; spad is linear
        // in r when Ns = 1 or Ns is a multiple of 16
        const int base = (tau - m) * P + m;
        cta_sync(nthr);
        if (Ns == 1 || (Ns & 15) == 0) {
          const int wr0 = spad(base) * C + c;
          const int wrr = (Ns + (Ns >> 4)) * C;
#pragma unroll
          for (int r = 0; r < P; ++r) sm[wr0 + r * wrr] = v[r];
        } else {
#pragma unroll
          for (int r = 0; r < P; ++r) sm[spad(base + r * Ns) * C + c] = v[r];
        }
        cta_sync(nthr);
        if ((TPT & 15) == 0) {
#pragma unroll
          for (int q = 0; q < P; ++q) v[q] = sm[rd0 + q * rdq];
        } else {
#pragma unroll
          for (int q = 0; q < P; ++q) v[q] = sm[spad(tau + TPT * q) * C + c];
        }
      }
      Ns *= P;
    }
    if constexpr (P >= 4) {
      if (rl == 1) last_small_stage<P, 2, DIR>(v, tau, TPT, tw, tws);
    }
    if constexpr (P >= 8) {
      if (rl == 2) last_small_stage<P, 4, DIR>(v, tau, TPT, tw, tws);
    }
    if constexpr (P >= 16) {
      if (rl == 3) last_small_stage<P, 8, DIR>(v, tau, TPT, tw, tws);
    }
  }
}

}  // namespace grf
