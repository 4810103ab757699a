// Device bodies of the FP32 passes, shared by the per-pass kernels
// (fft_kernels.cu) and the persistent uneven-batch kernel (batch.cu).  Each
// body takes its tile coordinates and the number of threads taking part, so a
// persistent CTA can run a tile that needs fewer threads than it has.
//
#pragma once
#include "kernels.h"
#include "fft_core.cuh"

namespace grf {

// ---------------------------------------------------------------------------
// Half-spectrum helpers
// ---------------------------------------------------------------------------

// Column index of a plane of H (axis 1 is the transform axis) -> (kmid, kd).
struct ColGeom {
  int kmid, kd;
};
GRF_DEV ColGeom col_geom(int col, const HalfGeom& g) {
  ColGeom r;
  r.kmid = col / (g.M + 1);
  r.kd = col - r.kmid * (g.M + 1);
  return r;
}

// Folded table index of (k1, kmid, kd): S depends on |p_i| only; the table is
// [kd][fmid][f1] so that lanes along axis 1 read consecutive entries.
GRF_DEV int fold_index(int k1, int kmid, int kd, const HalfGeom& g) {
  const int f1 = min(k1, g.N1 - k1);
  const int fm = min(kmid, g.Nmid - kmid);
  return (kd * (g.Nmid / 2 + 1) + fm) * (g.N1 / 2 + 1) + f1;
}

// The Philox key and the s_K table of the field at launch index z (a batch
// plan's launch maps z to its batch index and table; a plan's launch takes
// fields field0 + z with one table).
GRF_DEV uint64_t field_key(const HalfGeom& g, int64_t z) {
  const uint64_t seed = g.seed_ptr ? *g.seed_ptr : g.seed;
  return seed + (uint64_t)(g.zfield ? g.zfield[z] : g.field0 + z);
}
GRF_DEV const float* field_stab(const HalfGeom& g, int64_t z) { return g.stab + z * g.stab_zstride; }

// xi_K at (k1, kmid, kd) of field `field`.
GRF_DEV float2 xi_at(int k1, int kmid, int kd, int64_t field, const HalfGeom& g) {
  return alg2_xi_grid(k1, kmid, kd, g.N1, g.Nmid, g.M, g.seed + (uint64_t)(g.field0 + field), g.trig);
}

// Deterministic CTA sum of three doubles: warp shuffles, then warp 0 in order.
GRF_DEV void block_sum3(double v0, double v1, double v2, double* out3, double* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_down_sync(0xffffffffu, v0, o);
    v1 += __shfl_down_sync(0xffffffffu, v1, o);
    v2 += __shfl_down_sync(0xffffffffu, v2, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    scratch[3 * w] = v0;
    scratch[3 * w + 1] = v1;
    scratch[3 * w + 2] = v2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) {
      a += scratch[3 * i];
      b += scratch[3 * i + 1];
      c += scratch[3 * i + 2];
    }
    out3[0] = a;
    out3[1] = b;
    out3[2] = c;
  }
}

// xi_K on a plane kd in {0, M} (Eq. conj): the member of {K, -K} with the larger
// row-major index keeps its normals, the other takes their conjugate, and a
// self-conjugate K takes z_re.  Out of line: the column pass needs it for two
// columns only, and inlined copies would crowd the registers of the others.
static __device__ __noinline__ float2 plane_xi(int k1, int kmid, int kd, int N1, int Nmid, int M, uint64_t key,
                                               const float2* trig) {
  const int nk1 = (N1 - k1) & (N1 - 1), nkm = (Nmid - kmid) & (Nmid - 1);
  const int row = k1 * Nmid + kmid, nrow = nk1 * Nmid + nkm;
  const bool own = row >= nrow;
  const float2 z = alg2_normals_grid(own ? k1 : nk1, own ? kmid : nkm, kd, N1, Nmid, M, key, trig);
  if (row == nrow) return make_float2(z.x, 0.f);
  const float r2 = 0.70710678118654752440f;
  return make_float2(z.x * r2, own ? z.y * r2 : -z.y * r2);
}

// Normals (z_re, z_im) of Algorithm 2 for the entries (k1 = tau + TPT q, kmid, kd)
// of this thread (TPT P = N1).  Rows k1 and k1 + N1/2 share one Philox call
// (words 0,1 and 2,3), and they are this thread's entries q and q + P/2: each
// call feeds two of the thread's own entries, whatever the layout.
template <int P>
GRF_DEV void alg2_column_normals(float2 (&v)[P], int tau, int TPT, int kmid, int kd, const HalfGeom& g,
                                 uint64_t key) {
  // row k1 = tau + TPT i (i < P/2) lies below N1/2: its call is (k1 Nmid + kmid)(M + 1) + kd
  const uint64_t stride = (uint64_t)TPT * (uint64_t)g.Nmid * (uint64_t)(g.M + 1);
  uint64_t call = ((uint64_t)tau * (uint64_t)g.Nmid + (uint64_t)kmid) * (uint64_t)(g.M + 1) + (uint64_t)kd;
#pragma unroll
  for (int i = 0; i < P / 2; ++i, call += stride) {
    const u32x4 w = philox_call(call, 0u, key);
    v[i] = box_muller(w.x, w.y, g.trig);
    v[i + P / 2] = box_muller(w.z, w.w, g.trig);
  }
}

// ---------------------------------------------------------------------------
// Column pass
// ---------------------------------------------------------------------------

// Element (pos, col) of a plane in the tiled layout [pos / T][col][pos % T].
GRF_DEV int64_t col_offset(const ColArgs& a, int pos, int col) {
  return (int64_t)(pos >> a.logT) * (a.ncols << a.logT) + ((int64_t)col << a.logT) + (pos & (a.T - 1));
}

// Column `col` of the pass through its transforms: v[q] holds entry
// pos = tau + TPT q.  `base` is the offset of the column's plane and field.
// LN, CC: a compile-time transform length 2^LN and CC columns per CTA (see
// pass_kernels.cuh); 0 takes them from the launch descriptor.
template <int P, int SRC, int MODE, int LN = 0>
GRF_DEV void col_transform(const ColArgs& a, int col, bool valid, int64_t field, int64_t base, int tau, int c,
                           int C, int nthr, float2* sm, float2 (&v)[P], ColGeom& cg) {
  const int N = LN ? (1 << LN) : a.N;
  const int logN = LN ? LN : a.logN;
  const int TPT = N / P;
  cg = ColGeom{0, 0};
  if (SRC == COL_NOISE || MODE == COL_FWD_SCALE_INV || MODE == COL_FWD_ADJ) cg = col_geom(valid ? col : 0, a.g);

  if constexpr (SRC == COL_NOISE) {
    const HalfGeom& g = a.g;
    const uint64_t key = field_key(g, field);
    // s_K of this column: the folded table row (kd, fmid) is contiguous along axis 1
    const float* srow =
        field_stab(g, field) + (cg.kd * (g.Nmid / 2 + 1) + min(cg.kmid, g.Nmid - cg.kmid)) * (g.N1 / 2 + 1);
    alg2_column_normals<P>(v, tau, TPT, cg.kmid, cg.kd, g, key);
    // s_K read after the normals: the loads do not hold registers during the draw
    float s[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int k1 = tau + TPT * q;
      s[q] = __ldg(srow + min(k1, g.N1 - k1));
    }
    const float r2 = 0.70710678118654752440f;
    if (cg.kd != 0 && cg.kd != g.M) {
#pragma unroll
      for (int q = 0; q < P; ++q) v[q] = cscale(v[q], s[q] * r2);
    } else {
      // planes kd in {0, M}: conjugate pairs (Eq. conj) and the self-conjugate
      // points, out of line (2 of the M + 1 columns take this branch)
#pragma unroll
      for (int q = 0; q < P; ++q)
        v[q] = cscale(plane_xi(tau + TPT * q, cg.kmid, cg.kd, g.N1, g.Nmid, g.M, key, g.trig), s[q]);
    }
    if (!valid) {
#pragma unroll
      for (int q = 0; q < P; ++q) v[q] = make_float2(0.f, 0.f);
    }
  } else {
#pragma unroll
    for (int q = 0; q < P; ++q)
      v[q] = valid ? __ldcg(a.in + base + col_offset(a, tau + TPT * q, col)) : make_float2(0.f, 0.f);
  }

  if constexpr (MODE == COL_INV) {
    fft_core<P, +1>(v, sm, tau, c, C, N, logN, a.tw, a.tws, nthr);
  } else {
    fft_core<P, -1>(v, sm, tau, c, C, N, logN, a.tw, a.tws, nthr);
  }

  if constexpr (MODE == COL_FWD_SCALE_INV) {
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int k1 = tau + TPT * q;
      const float s = valid ? __ldg(a.g.stab + fold_index(k1, cg.kmid, cg.kd, a.g)) * a.g.alg1_scale : 0.f;
      v[q] = cscale(v[q], s);
    }
    fft_core<P, +1>(v, sm, tau, c, C, N, logN, a.tw, a.tws, nthr);
  }
}

// Pair mode (a.zpair), the last column pass before the c2r pass: one CTA
// takes C column pairs of plane `by` of field `bz`.  Slot p <= M/2 takes the
// columns kd = p and kd = M - p and writes, instead of X, the sequence the
// M-point inverse FFT of the c2r split consumes:
//   Z[p]     = (X[p] + conj X[M-p]) + i w (X[p] - conj X[M-p]),   w = e^{2 pi i p / N_d}
//   Z[M - p] = conj(X[p] + conj X[M-p]) + i conj(w (X[p] - conj X[M-p]))
// (the second is the first with p -> M - p, since e^{2 pi i (M-p)/N_d} = -conj w).
// Pair 0 (columns 0 and M) gives Z[0] only and pair M/2 is one column.  Z[k]
// lands where X[k] was (k < M; the slot of k = M is left unused), so the pass
// may run in place.  X of column p waits in shared memory, after the
// transform's exchange buffer, in a slot private to each thread
// (col_pair_smem_bytes), while column M - p is transformed.
//
// The indices of the pair are formed afresh after each transform (from the
// special registers in the per-pass kernels), so that nothing but the
// transform's own state is live while it runs.
struct CtaCoordsHW {  // per-pass kernels: blockIdx and threadIdx, re-read on each use
  GRF_DEV int bx() const { unsigned r; asm volatile("mov.u32 %0, %%ctaid.x;" : "=r"(r)); return (int)r; }
  GRF_DEV int by() const { unsigned r; asm volatile("mov.u32 %0, %%ctaid.y;" : "=r"(r)); return (int)r; }
  GRF_DEV int64_t bz() const { unsigned r; asm volatile("mov.u32 %0, %%ctaid.z;" : "=r"(r)); return (int64_t)r; }
  GRF_DEV int tid() const { unsigned r; asm volatile("mov.u32 %0, %%tid.x;" : "=r"(r)); return (int)r; }
};
struct CtaCoordsVal {  // persistent kernels: the tile's coordinates as values
  int x, y;
  int64_t z;
  GRF_DEV int bx() const { return x; }
  GRF_DEV int by() const { return y; }
  GRF_DEV int64_t bz() const { return z; }
  GRF_DEV int tid() const { return (int)threadIdx.x; }
};

struct PairIdx {
  int c, tau, p, ca, cb;
  bool valid;
  int64_t field, base;
};
template <int CC, class Coords>
GRF_DEV PairIdx pair_idx(const ColArgs& a, const Coords& co) {
  PairIdx r;
  const int C = CC ? CC : a.C;
  const int t = co.tid();
  r.c = t & (C - 1);
  r.tau = t / C;
  r.p = co.bx() * C + r.c;
  r.valid = r.p <= a.g.M / 2;
  r.ca = r.valid ? r.p : 0;
  r.cb = r.valid ? a.g.M - r.p : 0;
  r.field = co.bz();
  r.base = r.field * a.bstride + (int64_t)co.by() * a.ostride;
  return r;
}

template <int P, int SRC, int MODE, int LN = 0, int CC = 0, class Coords>
GRF_DEV void col_body_pair(const ColArgs& a, const Coords& co, int nthr_rt, float2* sm) {
  static_assert(MODE == COL_INV || MODE == COL_FWD_SCALE_INV, "pair mode ends an inverse pass");
  const int N = LN ? (1 << LN) : a.N;
  const int C = CC ? CC : a.C;
  const int nthr = (LN && CC) ? CC * (1 << LN) / P : nthr_rt;
  const int TPT = N / P;
  float2 v[P];
  ColGeom cg;
  if constexpr (SRC == COL_LOAD && MODE == COL_INV && P <= 8) {
    // loaded pair (3-D axis 2): both columns are read before either is
    // transformed (2 P complex values fit in the registers at P <= 8), so the
    // second column's loads overlap the first transform
    const int logN = LN ? LN : a.logN;
    float2 vb[P];
    {
      const PairIdx x = pair_idx<CC>(a, co);
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int pos = x.tau + TPT * q;
        v[q] = x.valid ? __ldcg(a.in + x.base + col_offset(a, pos, x.ca)) : make_float2(0.f, 0.f);
        vb[q] = x.valid ? __ldcg(a.in + x.base + col_offset(a, pos, x.cb)) : make_float2(0.f, 0.f);
      }
    }
    fft_core<P, +1>(v, sm, co.tid() / C, co.tid() & (C - 1), C, N, logN, a.tw, a.tws, nthr);
    float2* stash = sm + (size_t)spad(N) * C + co.tid();
#pragma unroll
    for (int q = 0; q < P; ++q) stash[q * nthr] = v[q];
#pragma unroll
    for (int q = 0; q < P; ++q) v[q] = vb[q];
    fft_core<P, +1>(v, sm, co.tid() / C, co.tid() & (C - 1), C, N, logN, a.tw, a.tws, nthr);
  } else {
    {
      const PairIdx x = pair_idx<CC>(a, co);
      col_transform<P, SRC, MODE, LN>(a, x.ca, x.valid, x.field, x.base, x.tau, x.c, C, nthr, sm, v, cg);
    }
    float2* stash = sm + (size_t)spad(N) * C + co.tid();
#pragma unroll
    for (int q = 0; q < P; ++q) stash[q * nthr] = v[q];
    {
      // pair M/2 is one column: its second transform only keeps the CTA's
      // barriers in step (an in-place pass has already replaced its input)
      const PairIdx x = pair_idx<CC>(a, co);
      col_transform<P, SRC, MODE, LN>(a, x.cb, x.valid && x.ca != x.cb, x.field, x.base, x.tau, x.c, C, nthr,
                                          sm, v, cg);
    }
  }
  const PairIdx x = pair_idx<CC>(a, co);
  if (!x.valid) return;
  float2* out = a.out + x.base;
  const float2 w = __ldg(a.twz + x.p);
  const float2* stash = sm + (size_t)spad(N) * C + co.tid();
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int64_t oa = col_offset(a, x.tau + TPT * q, x.ca);
    const float2 xa = stash[q * nthr];
    const float2 xb = x.ca == x.cb ? xa : v[q];
    const float2 A = make_float2(xa.x + xb.x, xa.y - xb.y);
    const float2 B = make_float2(xa.x - xb.x, xa.y + xb.y);
    const float2 wB = cmul(w, B);
    out[oa] = make_float2(A.x - wB.y, A.y + wB.x);
    if (x.p != 0 && x.ca != x.cb) out[col_offset(a, x.tau + TPT * q, x.cb)] = make_float2(A.x + wB.y, wB.x - A.y);
  }
}

// One CTA: C columns of plane `by` of field `bz`, X stored (or, for the
// adjoint, reduced).
template <int P, int SRC, int MODE, int LN = 0, int CC = 0>
GRF_DEV void col_body(const ColArgs& a, int bx, int by, int64_t bz, int64_t blk, int nthr_rt, float2* sm) {
  const int C = CC ? CC : a.C;
  const int nthr = (LN && CC) ? CC * (1 << LN) / P : nthr_rt;
  const int t = threadIdx.x;
  const int c = t & (C - 1);
  const int tau = t / C;
  const int TPT = (LN ? (1 << LN) : a.N) / P;
  const int64_t field = bz;
  const int64_t base = field * a.bstride + (int64_t)by * a.ostride;
  float2 v[P];
  ColGeom cg;

  const int col = bx * C + c;
  const bool valid = col < a.ncols;
  col_transform<P, SRC, MODE, LN>(a, col, valid, field, base, tau, c, C, nthr, sm, v, cg);

  if constexpr (MODE == COL_FWD_ADJ) {
    // v[q] = G^ at K = (k1, kmid, kd).  Sum w_K d_theta s_K Re(xi_K conj G^_K).
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    if (valid) {
      const float w = (cg.kd == 0 || cg.kd == a.g.M) ? 1.f : 2.f;
      const int hsz = (a.g.N1 / 2 + 1) * (a.g.Nmid / 2 + 1) * (a.g.M + 1);
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int k1 = tau + TPT * q;
        const int fi = fold_index(k1, cg.kmid, cg.kd, a.g);
        const float2 xi = xi_at(k1, cg.kmid, cg.kd, field, a.g);
        const float re = w * fmaf(xi.x, v[q].x, xi.y * v[q].y);
        a0 = fmaf(re, __ldg(a.g.stab + fi), a0);
        a1 = fmaf(re, __ldg(a.g.dstab + fi), a1);
        a2 = fmaf(re, __ldg(a.g.dstab + hsz + fi), a2);
      }
    }
    double* scratch = reinterpret_cast<double*>(sm);
    block_sum3((double)a0 * a.g.inv_sigma, (double)a1, (double)a2, a.partial + 3 * blk, scratch);
    return;
  }

  if (valid) {
    if (a.pitch3) {  // padded rows for the plane path's sub-plane kernel
      const int64_t scol = (int64_t)cg.kmid * a.pitch3 + cg.kd, rstride = (int64_t)a.g.Nmid * a.pitch3;
#pragma unroll
      for (int q = 0; q < P; ++q) a.out[base + (int64_t)(tau + TPT * q) * rstride + scol] = v[q];
    } else {
#pragma unroll
      for (int q = 0; q < P; ++q) a.out[base + col_offset(a, tau + TPT * q, col)] = v[q];
    }
  }
}

// ---------------------------------------------------------------------------
// Row pass
// ---------------------------------------------------------------------------

// Offset of row g, entry 0 in a half-spectrum array with row tile T (a power of 2):
// (g / T) * ((M + 1) T) + (g % T); entry k adds k T.
GRF_DEV int64_t hrow_base(int64_t g, int M, int logT) {
  return ((g >> logT) * (int64_t)(M + 1) << logT) + (g & ((1 << logT) - 1));
}

// Z[k] of the c2r split from X[k] and X[M - k] (both in shared memory).
GRF_DEV float2 c2r_pre(float2 X, float2 Y, float2 w) {
  // A = X + conj Y, B = X - conj Y, Z = A + i w B
  const float2 A = make_float2(X.x + Y.x, X.y - Y.y);
  const float2 B = make_float2(X.x - Y.x, X.y + Y.y);
  const float2 wB = cmul(w, B);
  return make_float2(A.x - wB.y, A.y + wB.x);
}

// X[k] of the r2c split from Zf[k] and Zf[M - k]: 1/2 (A - i conj(w) B) with
// A = Zk + conj Zmk, B = Zk - conj Zmk, w = exp(2 pi i k / N).
GRF_DEV float2 r2c_post(float2 Zk, float2 Zmk, float2 w) {
  const float2 A = make_float2(Zk.x + Zmk.x, Zk.y - Zmk.y);
  const float2 B = make_float2(Zk.x - Zmk.x, Zk.y + Zmk.y);
  const float2 wB = cmulc(B, w);  // B * conj(w)
  return make_float2(0.5f * (A.x + wB.y), 0.5f * (A.y - wB.x));
}

// LN, CC: a compile-time length M = 2^LN and CC rows per CTA (see
// pass_kernels.cuh); 0 takes them from the launch descriptor.
// BZ: the output pointer comes from a.zout (1, a batch plan's launch), from
// a.outR (0), or whichever is set (-1).
template <int P, int SRC, int MODE, int LN = 0, int CC = 0, int TT = 0, int BZ = -1>
GRF_DEV void row_body(const RowArgs& a, int64_t bx, int nthr_rt, float2* sm) {
  const int C = CC ? CC : a.C;
  const int nthr = (LN && CC) ? CC * (1 << LN) / P : nthr_rt;
  const int t = threadIdx.x;
  const int c = t & (C - 1);
  const int tau = t / C;
  const int M = LN ? (1 << LN) : a.M;
  const int logM = LN ? LN : a.logM;
  const int N = 2 * M;
  const int TPT = M / P;
  const int64_t g = bx * C + c;
  const bool valid = g < a.nrows;
  const int64_t field = valid ? g / a.rows_per_field : 0;
  const int64_t rowf = valid ? g - field * a.rows_per_field : 0;
  float2 v[P];

  if constexpr (MODE == ROW_C2R && SRC == ROW_LOAD_Z) {
    // Z[0..M-1] of the c2r split, formed by the last column pass: straight
    // into the M-point inverse FFT.
    // TT: a compile-time tile (the loads then differ by constant offsets)
    const int logT = TT ? ilog2c(TT) : a.logT;
    const float2* src = a.inH + hrow_base(valid ? g : 0, M, logT);
#pragma unroll
    for (int q = 0; q < P; ++q)
      v[q] = valid ? __ldcg(src + ((int64_t)(tau + TPT * q) << logT)) : make_float2(0.f, 0.f);
    fft_core<P, +1>(v, sm, tau, c, C, M, logM, a.twM, a.tws, nthr);
    if (valid) {
      // (the row's field is formed only for a batch plan's launch)
      const bool bz = BZ < 0 ? a.zout != nullptr : BZ == 1;
      float2* o = reinterpret_cast<float2*>(
          bz ? a.zout[g / a.rows_per_field] + (g % a.rows_per_field) * N : a.outR + g * N);
#pragma unroll
      for (int q = 0; q < P; ++q) o[tau + TPT * q] = v[q];
    }
    return;
  } else if constexpr (MODE == ROW_C2R) {
    // ROW_NOISE_H (d = 1, one row per field): stage X[0..M] of every row of
    // the CTA in shared memory, then split into Z.
    const uint64_t key = field_key(a.g, field);
    const float* stab = field_stab(a.g, field);
    float2 xm = make_float2(0.f, 0.f);
    if (valid) {
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int k = tau + TPT * q;
        v[q] = cscale(alg2_xi_1d(k, M, key, a.g.trig), __ldg(stab + k));
      }
      if (tau == 0) xm = cscale(alg2_xi_1d(M, M, key, a.g.trig), __ldg(stab + M));
    } else {
#pragma unroll
      for (int q = 0; q < P; ++q) v[q] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < P; ++q) sm[spad(tau + TPT * q) * C + c] = v[q];
    if (tau == 0) sm[spad(M) * C + c] = xm;
    cta_sync(nthr);
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int k = tau + TPT * q;
      v[q] = c2r_pre(sm[spad(k) * C + c], sm[spad(M - k) * C + c], __ldg(a.twN + k));
    }
    if constexpr (P < 16) cta_sync(nthr);
    fft_core<P, +1>(v, sm, tau, c, C, M, logM, a.twM, a.tws, nthr);
    if (valid) {
      float2* o = reinterpret_cast<float2*>(a.zout ? a.zout[field] + rowf * N : a.outR + g * N);
#pragma unroll
      for (int q = 0; q < P; ++q) o[tau + TPT * q] = v[q];
    }
    return;
  } else {
    // Forward r2c of a real row: z[m] = x[2m] + i x[2m+1].
    const uint64_t key = a.g.seed + (uint64_t)(a.g.field0 + field);
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int m = tau + TPT * q;
      float2 z = make_float2(0.f, 0.f);
      if (valid) {
        if constexpr (SRC == ROW_LOAD_REAL) {
          z = reinterpret_cast<const float2*>(a.inR + g * N)[m];
        } else {  // ROW_NOISE_REAL (Algorithm 1): flat index of the point
          z = alg1_normal_pair((uint64_t)(rowf * N + 2 * m), key, a.g.trig);
        }
      }
      v[q] = z;
    }
    fft_core<P, -1>(v, sm, tau, c, C, M, logM, a.twM, a.tws, nthr);
    cta_sync(nthr);
#pragma unroll
    for (int q = 0; q < P; ++q) sm[spad(tau + TPT * q) * C + c] = v[q];
    cta_sync(nthr);
    float2 X[P];
    float2 XM = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int k = tau + TPT * q;
      const float2 Zmk = sm[spad((M - k) & (M - 1)) * C + c];
      X[q] = r2c_post(v[q], Zmk, __ldg(a.twN + k));
    }
    if (tau == 0) XM = make_float2(v[0].x - v[0].y, 0.f);  // k = M: Re Z0 - Im Z0

    if constexpr (MODE == ROW_R2C) {
      if (valid) {
        const int64_t hb = hrow_base(g, M, a.logT);
#pragma unroll
        for (int q = 0; q < P; ++q) a.outH[hb + ((int64_t)(tau + TPT * q) << a.logT)] = X[q];
        if (tau == 0) a.outH[hb + ((int64_t)M << a.logT)] = XM;
      }
      return;
    } else if constexpr (MODE == ROW_R2C_SCALE_C2R) {
      // 1-D Algorithm 1: A = s_K DFT(z) / sqrt(N_tot), then c2r.
      const float sc = a.g.alg1_scale;
#pragma unroll
      for (int q = 0; q < P; ++q) X[q] = cscale(X[q], __ldg(a.g.stab + tau + TPT * q) * sc);
      if (tau == 0) XM = cscale(XM, __ldg(a.g.stab + M) * sc);
      cta_sync(nthr);
#pragma unroll
      for (int q = 0; q < P; ++q) sm[spad(tau + TPT * q) * C + c] = X[q];
      if (tau == 0) sm[spad(M) * C + c] = XM;
      cta_sync(nthr);
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int k = tau + TPT * q;
        v[q] = c2r_pre(X[q], sm[spad(M - k) * C + c], __ldg(a.twN + k));
      }
      if constexpr (P < 16) cta_sync(nthr);
      fft_core<P, +1>(v, sm, tau, c, C, M, logM, a.twM, a.tws, nthr);
      if (valid) {
        float2* o = reinterpret_cast<float2*>(a.outR + g * N);
#pragma unroll
        for (int q = 0; q < P; ++q) o[tau + TPT * q] = v[q];
      }
      return;
    } else {  // ROW_R2C_ADJ: 1-D adjoint, one row per field
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
      if (valid) {
#pragma unroll
        for (int q = 0; q <= P; ++q) {
          int k;
          float2 G;
          if (q < P) {
            k = tau + TPT * q;
            G = X[q];
          } else {
            if (tau != 0) break;
            k = M;
            G = XM;
          }
          const float w = (k == 0 || k == M) ? 1.f : 2.f;
          const float2 xi = alg2_xi_1d(k, M, key, a.g.trig);
          const float re = w * fmaf(xi.x, G.x, xi.y * G.y);
          a0 = fmaf(re, __ldg(a.g.stab + k), a0);
          a1 = fmaf(re, __ldg(a.g.dstab + k), a1);
          a2 = fmaf(re, __ldg(a.g.dstab + (M + 1) + k), a2);
        }
      }
      // per-row deterministic sum over the TPT threads of the row
      double* sd = reinterpret_cast<double*>(sm);
      cta_sync(nthr);
      sd[3 * t] = (double)a0 * a.g.inv_sigma;
      sd[3 * t + 1] = a1;
      sd[3 * t + 2] = a2;
      cta_sync(nthr);
      if (tau == 0 && valid) {
        double s0 = 0, s1 = 0, s2 = 0;
        for (int u = 0; u < TPT; ++u) {
          const int tt = u * C + c;
          s0 += sd[3 * tt];
          s1 += sd[3 * tt + 1];
          s2 += sd[3 * tt + 2];
        }
        a.partial[3 * g] = s0;
        a.partial[3 * g + 1] = s1;
        a.partial[3 * g + 2] = s2;
      }
      return;
    }
  }
}

// ---------------------------------------------------------------------------
// Four-step c2r for long 1-D grids
// ---------------------------------------------------------------------------

// X[k] = s_k xi_k of a 1-D field (xi real at the self-conjugate k = 0 and k = M).
GRF_DEV float2 x1d(int k, int M, const float* __restrict__ stab, uint64_t key, const float2* trig) {
  return cscale(alg2_xi_1d(k, M, key, trig), __ldg(stab + k));
}

template <int P>
GRF_DEV void fourstep1_body(const FourStepArgs& a, int bx, int64_t bz, int nthr, float2* sm) {
  const int C = a.C;
  const int t = threadIdx.x;
  const int c = t & (C - 1);
  const int tau = t / C;
  const int TPT = a.B / P;
  const int k1 = bx * C + c;  // < A: C divides A
  const int64_t field = bz;
  const uint64_t key = (a.seed_ptr ? *a.seed_ptr : a.seed) + (uint64_t)(a.zfield ? a.zfield[field] : a.field0 + field);
  const float* stab = a.stab + field * a.stab_zstride;
  float2 v[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int k = k1 + a.A * (tau + TPT * q);
    const int mk = a.M - k;  // k = 0 pairs with X[M]
    v[q] = c2r_pre(x1d(k, a.M, stab, key, a.trig), x1d(mk, a.M, stab, key, a.trig), __ldg(a.twN + k));
  }
  fft_core<P, +1>(v, sm, tau, c, C, a.B, a.logB, a.twB, a.tws, nthr);
  float2* Y = a.Y + field * (int64_t)a.M + ((k1 >> a.logT) * (int64_t)a.B << a.logT) + (k1 & (a.T - 1));
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int n2 = tau + TPT * q;
    Y[(int64_t)n2 << a.logT] = cmul(v[q], __ldg(a.twM + n2 * k1));
  }
}

// Stage 1 with mirror-closed columns: Z[k] needs X[k] and X[M - k], and the
// entries of column k1 mirror those of column A - k1 (M - k1 - A k2 =
// (A - k1) + A (B - 1 - k2); column 0 mirrors itself, M - A k2 = A (B - k2),
// with X[M] for k2 = 0; column A/2 mirrors itself too).  A CTA takes H = C/2
// pairs p in [bx H, bx H + H): slot c < H holds column p = bx H + c, slot
// c >= H column A - p' with p' = bx H + (C - 1 - c) (ascending in c), so slot
// c and slot C - 1 - c are mirrors.  Each X is drawn once, staged in shared
// memory, and read back by the thread that forms its mirror's Z.  Y is written
// with tile T = H (a.T), the second half's run straddling two tiles.
// LB, CC != 0: the transform length B = 2^LB and CC columns per CTA as
// constants (256 threads).
template <int P, int LB = 0, int CC = 0>
GRF_DEV void fourstep1_pair_body(const FourStepArgs& a, int bx, int64_t bz, int nthr_rt, float2* sm) {
  constexpr bool spec = LB && CC;
  const int B = spec ? (1 << LB) : a.B;
  const int logB = spec ? LB : a.logB;
  const int C = spec ? CC : a.C, H = C / 2;
  const int nthr = spec ? CC * (1 << LB) / P : nthr_rt;
  const int t = threadIdx.x;
  const int c = t & (C - 1);
  const int tau = t / C;
  const int TPT = B / P;
  const int half = a.A / 2;
  int k1;
  bool valid;
  if (c < H) {
    k1 = bx * H + c;
    valid = k1 <= half;
  } else {
    const int p = bx * H + (C - 1 - c);
    k1 = a.A - p;
    valid = p >= 1 && p < half;
  }
  if (!valid) k1 = 0;
  const int64_t field = bz;
  const uint64_t key = (a.seed_ptr ? *a.seed_ptr : a.seed) + (uint64_t)(a.zfield ? a.zfield[field] : a.field0 + field);
  const float* stab = a.stab + field * a.stab_zstride;
  const float* srow = a.stabT + field * a.stabT_zstride + (int64_t)k1 * B;  // s_{k1 + A k2} at k2
  // X of this slot's entries k = k1 + A k2, k2 = tau + TPT q, staged as [c][k2]
  // with a pitch of B + 16 / C (C < 16) or B + 1: a half warp (16 / C values of
  // tau for each of the C slots) then writes and reads 16 distinct bank pairs
  const int pitch = B + (C < 16 ? 16 / C : 1);
  float2 v[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int k2 = tau + TPT * q;
    const int k = k1 + a.A * k2;
    v[q] = valid ? cscale(alg2_xi_1d(k, a.M, key, a.trig), __ldg(srow + k2)) : make_float2(0.f, 0.f);
  }
  cta_sync(nthr);  // the exchange buffer may still be read by a previous use
#pragma unroll
  for (int q = 0; q < P; ++q) sm[c * pitch + tau + TPT * q] = v[q];
  cta_sync(nthr);
  // Z[k] from X[k] and its mirror; e^{2 pi i k / N} = e^{2 pi i k1 / N} e^{2 pi i k2 / (2B)}
  const bool self = k1 == 0 || k1 == half;
  const int mc = self ? c : C - 1 - c;
  const float2 wk1 = __ldg(a.twN + k1);
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int k2 = tau + TPT * q;
    float2 xm;
    if (k1 == 0) xm = k2 == 0 ? x1d(a.M, a.M, stab, key, a.trig) : sm[mc * pitch + B - k2];
    else xm = sm[mc * pitch + B - 1 - k2];
    v[q] = c2r_pre(v[q], xm, cmul(wk1, __ldg(a.tw2B + k2)));
  }
  fft_core<P, +1>(v, sm, tau, c, C, B, logB, a.twB, a.tws, nthr);
  if (!valid) return;
  float2* Y = a.Y + field * (int64_t)a.M + ((k1 >> a.logT) * (int64_t)B << a.logT) + (k1 & (a.T - 1));
#pragma unroll
  for (int q = 0; q < P; ++q) {
    // e^{2 pi i x / M}, x = n2 k1 < M, as e^{2 pi i (x >> log B) / A} e^{2 pi i (x mod B) / M}
    const int n2 = tau + TPT * q;
    const int x = n2 * k1;
    const float2 w = cmul(__ldg(a.twMA + (x >> logB)), __ldg(a.twM + (x & (B - 1))));
    Y[(int64_t)n2 << a.logT] = cmul(v[q], w);
  }
}

// LA, CC != 0: the transform length A = 2^LA and CC columns per CTA as
// constants (256 threads).
template <int P, int LA = 0, int CC = 0>
GRF_DEV void fourstep2_body(const FourStepArgs& a, int bx, int64_t bz, int nthr_rt, float2* sm) {
  constexpr bool spec = LA && CC;
  const int A = spec ? (1 << LA) : a.A;
  const int logA = spec ? LA : a.logA;
  const int C = spec ? CC : a.C;
  const int nthr = spec ? CC * (1 << LA) / P : nthr_rt;
  const int t = threadIdx.x;
  const int c = t & (C - 1);
  const int tau = t / C;
  const int TPT = A / P;
  const int n2 = bx * C + c;  // < B: C divides B
  const int64_t field = bz;
  const float2* Y = a.Yin + field * (int64_t)a.M + ((int64_t)n2 << a.logT);
  float2 v[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int k1 = tau + TPT * q;
    v[q] = __ldcg(Y + ((k1 >> a.logT) * (int64_t)a.B << a.logT) + (k1 & (a.T - 1)));
  }
  fft_core<P, +1>(v, sm, tau, c, C, A, logA, a.twA, a.tws, nthr);
  float2* o = reinterpret_cast<float2*>(a.zout ? a.zout[field] : a.out + field * (int64_t)a.N);
#pragma unroll
  for (int q = 0; q < P; ++q) o[n2 + (int64_t)a.B * (tau + TPT * q)] = v[q];
}

}  // namespace grf
