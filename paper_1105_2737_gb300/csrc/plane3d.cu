// The 3-D plane path of Algorithm 2 (FP32): pass 1 (plane3d_noise.cuh) and
// pass 2, the sub-plane kernel below, with their launchers.  Against the
// three-pass form (noise + axis 1, axis 2 in place, c2r) the intermediate half
// spectrum crosses HBM once instead of twice.
//
// Pass 2 takes one sub-plane (field, j1, s) of Q x (M + 1) complex values
// (row pitch S3 = M + 2) per CTA:
//   1. one bulk copy (cp.async.bulk, the Tensor Memory Accelerator) brings the
//      contiguous sub-plane into shared memory, completed on an mbarrier; the
//      wait is bounded (iterations and time) and a wait that runs out stores
//      GRF_ERR_TIMEOUT in the plan's status word;
//   2. the inverse FFTs of length Q along k' of its M + 1 columns, in place,
//      in batches of CB columns (the transposition is the shared-memory read
//      along a column);
//   3. per row j' (the axis-2 output j2 = s + R j'): the c2r split
//      Z[k] = (X[k] + conj X[M-k]) + i e^{2 pi i k / N3} (X[k] - conj X[M-k]),
//      k < M, the M-point inverse FFT, the N3 = 2M reals staged back into the
//      row's own slot and written to the field by one bulk copy per row.
#include "grf.h"
#include "plane3d_noise.cuh"
#include "pass_kernels.cuh"
#include "tma.cuh"

namespace grf {

using namespace tma;

namespace {

__host__ __device__ constexpr int pow2_at_least(int x) { return x <= 1 ? 1 : 2 * pow2_at_least((x + 1) / 2); }

// Pass 2's shapes: one sub-plane (Q rows of pitch S3 = M + 2) per CTA, 256
// threads when two CTAs fit on an SM, else 512.
__host__ __device__ constexpr size_t plane3_sub_bytes(int Q, int M) { return (size_t)Q * (M + 2) * sizeof(float2); }
__host__ __device__ constexpr size_t plane3_xb_bytes(int Q, int M, int NT) {
  return sizeof(float2) * ((size_t)(Q + Q / 16) * (NT / (Q / 16)) > (size_t)(M + M / 16) * (NT / (M / 16))
                               ? (size_t)(Q + Q / 16) * (NT / (Q / 16))
                               : (size_t)(M + M / 16) * (NT / (M / 16)));
}
__host__ __device__ constexpr int plane3_threads(int Q, int M) {
  return 2 * (128 + plane3_sub_bytes(Q, M) + plane3_xb_bytes(Q, M, 256) + 1024) <= 228 * 1024 ? 256 : 512;
}
__host__ __device__ constexpr size_t plane3_c2r_smem_bytes(int Q, int M) {
  return 128 + plane3_sub_bytes(Q, M) + plane3_xb_bytes(Q, M, plane3_threads(Q, M));
}

// One sub-plane `id` ((field N1 + j1) R + s) held in `sub`: the axis-2 inverse
// FFTs along k', the c2r rows, and one bulk store per row issued by threads
// t < RB (committed and waited for by the caller).
template <int LQ, int LM, int NT>
GRF_DEV void plane3_subplane(const PlaneArgs& pl, float2* sub, float2* xb, int64_t id) {
  constexpr int P = 16, Q = 1 << LQ, M = 1 << LM, S3 = M + 2;
  constexpr int TPC = Q / P, CB = NT / TPC;  // columns per batch
  constexpr int TPR = M / P, CR = NT / TPR;  // rows per batch
  constexpr int RB = CR < Q ? CR : Q;        // rows per batch that exist
  static_assert(Q % CR == 0 || CR > Q, "whole row batches");
  const int t = threadIdx.x;
  // axis 2: inverse FFTs of length Q along k' of the columns k3 = 0..M, in
  // place.  The planes k3 = 0 and k3 = M are Hermitian in (k1, k2), so after
  // axis 1 each of their columns has a real inverse DFT along k2 (and so along
  // k' for every residue s): they share one transform as X[k', 0] + i X[k', M]
  // (real part: column 0, imaginary part: column M).  That leaves M columns,
  // a whole number of batches when CB divides M; a remainder runs on the
  // fewest whole warps that hold it, the other warps going ahead.
  const float2* twQ = pl.tw + Q;
  constexpr int FULL = M / CB, REM = M - FULL * CB;
  // columns of the last call: a power of two >= REM whose threads fill whole warps
  constexpr int CREM = pow2_at_least(REM > 32 / TPC ? REM : 32 / TPC) < CB ? pow2_at_least(REM > 32 / TPC ? REM : 32 / TPC) : CB;
  static_assert((CREM & (CREM - 1)) == 0 && (CREM * TPC) % 32 == 0, "whole warps");
  for (int bi = 0; bi <= FULL; ++bi) {
    const int C = bi < FULL ? CB : CREM;
    const int nthr = C * TPC;
    if (bi == FULL) {
      __syncthreads();  // every warp has read the exchange buffer of the last full batch
      if (REM == 0 || t >= nthr) break;
    }
    const int c = t % C, tau = t / C;
    const int col = bi * CB + c;  // column 0 carries the planes k3 = 0 and k3 = M
    const bool valid = col < M;
    float2 v[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const float2* x = sub + (tau + TPC * q) * S3;
      if (col == 0) {
        const float2 a = x[0], b = x[M];
        v[q] = make_float2(a.x - b.y, a.y + b.x);  // a + i b
      } else {
        v[q] = valid ? x[col] : make_float2(0.f, 0.f);
      }
    }
    fft_core<P, +1>(v, xb, tau, c, C, Q, LQ, twQ, pl.tws, nthr);
    if (valid) {
#pragma unroll
      for (int q = 0; q < P; ++q) {
        float2* x = sub + (tau + TPC * q) * S3;
        if (col == 0) {
          x[0] = make_float2(v[q].x, 0.f);
          x[M] = make_float2(v[q].y, 0.f);
        } else {
          x[col] = v[q];
        }
      }
    }
  }
  __syncthreads();
  // axis 3: c2r split + M-point inverse FFT per row, rows back to the field by bulk copies
  const int R = pl.R;
  const int64_t fj = id / R;  // field N1 + j1
  const int s = (int)(id - fj * R);
  float* plane = pl.zout ? pl.zout[fj / pl.N1] + (fj % pl.N1) * (int64_t)pl.N2 * (2 * M)
                         : pl.out + fj * (int64_t)pl.N2 * (2 * M);
  const float2* twM = pl.tw + M;
  const float2* twN = pl.tw + 2 * M;
  for (int r0 = 0; r0 < Q; r0 += RB) {
    const int c = t % CR, tau = t / CR;
    const int row = r0 + (c < RB ? c : 0);
    float2 v[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int k = tau + TPR * q;
      v[q] = c2r_pre(sub[row * S3 + k], sub[row * S3 + M - k], __ldg(twN + k));
    }
    fft_core<P, +1>(v, xb, tau, c, CR, M, LM, twM, pl.tws, NT);
    if (c < RB) {
#pragma unroll
      for (int q = 0; q < P; ++q) sub[row * S3 + tau + TPR * q] = v[q];
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (t < RB) {
      const int rr = r0 + t;
      bulk_store(plane + (int64_t)(s + R * rr) * (2 * M), smem_addr(sub + rr * S3), (uint32_t)(M * sizeof(float2)));
    }
  }
}

// One slot: one CTA per sub-plane.
template <int LQ, int LM>
__global__ void __launch_bounds__(plane3_threads(1 << LQ, 1 << LM), 1) plane3_c2r_kernel(PlaneArgs pl) {
  constexpr int Q = 1 << LQ, M = 1 << LM, NT = plane3_threads(Q, M);
  constexpr int TPR = M / 16, CR = NT / TPR, RB = CR < Q ? CR : Q;
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
  float2* sub = reinterpret_cast<float2*>(smraw + 128);
  float2* xb = sub + (size_t)Q * (M + 2);
  const int t = threadIdx.x;
  const int64_t id = blockIdx.x;
  const uint32_t b0 = smem_addr(bar);
  if (t == 0) {
    mbar_init(b0);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bulk_load(smem_addr(sub), pl.ws + id * (int64_t)Q * (M + 2), (uint32_t)plane3_sub_bytes(Q, M), b0);
  }
  __syncthreads();
  const bool ok = mbar_wait(b0, 0);
  if (__syncthreads_or(!ok)) {
    if (t == 0) {
      atomicExch(pl.status, (int)GRF_ERR_TIMEOUT);
      mbar_wait(b0, 0);  // the copy still in flight, if it ever completes
    }
    __syncthreads();
    return;
  }
  plane3_subplane<LQ, LM, NT>(pl, sub, xb, id);
  if (t < RB) {
    bulk_commit();
    bulk_wait_read_all();
  }
}

template <int LQ, int LM>
cudaError_t c2r_t(const PlaneArgs& pl, int64_t nfields, cudaStream_t s) {
  constexpr int Q = 1 << LQ, M = 1 << LM;
  const size_t smem = plane3_c2r_smem_bytes(Q, M);
  auto k = plane3_c2r_kernel<LQ, LM>;
  cudaError_t e = prepare_kernel((const void*)k, plane3_threads(Q, M), smem);
  if (e != cudaSuccess) return e;
  const int64_t nsub = nfields * pl.N1 * pl.R;
  k<<<(unsigned)nsub, plane3_threads(Q, M), smem, s>>>(pl);
  return cudaGetLastError();
}

// (log2 Q, log2 M) with a compiled pass 2: Q in 16..128, M in 16..512, the
// shared memory within 227 KB.
constexpr bool plane3_supported(int LQ, int LM) {
  return LQ >= 4 && LQ <= 7 && LM >= 4 && LM <= 9 && plane3_c2r_smem_bytes(1 << LQ, 1 << LM) <= 227 * 1024;
}

template <int LQ, int LM>
cudaError_t c2r_dispatch_m(const PlaneArgs& pl, int64_t nfields, cudaStream_t s) {
  if constexpr (plane3_supported(LQ, LM)) return c2r_t<LQ, LM>(pl, nfields, s);
  return cudaErrorInvalidValue;
}

template <int LQ>
cudaError_t c2r_dispatch_q(int lm, const PlaneArgs& pl, int64_t nfields, cudaStream_t s) {
  switch (lm) {
    case 4: return c2r_dispatch_m<LQ, 4>(pl, nfields, s);
    case 5: return c2r_dispatch_m<LQ, 5>(pl, nfields, s);
    case 6: return c2r_dispatch_m<LQ, 6>(pl, nfields, s);
    case 7: return c2r_dispatch_m<LQ, 7>(pl, nfields, s);
    case 8: return c2r_dispatch_m<LQ, 8>(pl, nfields, s);
    case 9: return c2r_dispatch_m<LQ, 9>(pl, nfields, s);
    default: return cudaErrorInvalidValue;
  }
}

int lg(int x) {
  int r = 0;
  while ((1 << r) < x) ++r;
  return r;
}

bool pow2i(int x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace

int plane3_radix(int N1, int N2, int M) {
  if (!pow2i(N1) || !pow2i(N2) || !pow2i(M) || N1 < 2 || N1 > 1024) return 0;
  if (N1 < 256) {  // the column pass writes whole planes (R = 1) with padded rows
    const int LQ = lg(N2), LM = lg(M);
    if (!(LQ >= 4 && LQ <= 7 && LM >= 4 && LM <= 9)) return 0;
    return plane3_c2r_smem_bytes(N2, M) <= 227 * 1024 ? 1 : 0;
  }
  const int CC = 4096 / N1;
  int fallback = 0;
  // pass 1 writes runs of U = CC / R consecutive k3: at least 4 (32 bytes), or
  // its stores scatter over sectors and it runs up to twice as long
  for (int R = 1; R <= 16; R *= 2) {
    if (4 * R > CC || R > N2) break;
    const int Q = N2 / R;
    const int LQ = lg(Q), LM = lg(M);
    if (!(LQ >= 4 && LQ <= 7 && LM >= 4 && LM <= 9)) continue;
    if (plane3_c2r_smem_bytes(Q, M) > 227 * 1024) continue;
    if (plane3_threads(Q, M) == 256) return R;  // two CTAs per SM in pass 2
    if (!fallback) fallback = R;
  }
  return fallback;
}

size_t plane3_ws_entries(int N1, int N2, int M) { return (size_t)N1 * N2 * (M + 2); }

namespace {

template <int LN, int R>
cudaError_t noise_t(const ColArgs& a, const PlaneArgs& pl, int64_t nfields, cudaStream_t s) {
  constexpr int CC = 4096 >> LN;
  if constexpr (4 * R > CC) {
    return cudaErrorInvalidValue;
  } else {
    constexpr int U = CC / R;
    const size_t smem = plane3_noise_smem_bytes(1 << LN, CC);
    auto k = plane3_noise_kernel<LN, CC, R>;
    cudaError_t e = prepare_kernel((const void*)k, 256, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((pl.M + 1 + U - 1) / U), (unsigned)pl.Q, (unsigned)nfields);
    k<<<grid, 256, smem, s>>>(a, pl);
    return cudaGetLastError();
  }
}

template <int LN>
cudaError_t noise_ln(const ColArgs& a, const PlaneArgs& pl, int64_t nfields, cudaStream_t s) {
  switch (pl.R) {
    case 1: return noise_t<LN, 1>(a, pl, nfields, s);
    case 2: return noise_t<LN, 2>(a, pl, nfields, s);
    case 4: return noise_t<LN, 4>(a, pl, nfields, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_plane3_noise(const ColArgs& a, const PlaneArgs& pl, int64_t nfields, cudaStream_t s) {
  if (a.N != pl.N1 || pl.R < 1 || pl.Q * pl.R != pl.N2 || pl.S3 != pl.M + 2 || nfields < 1)
    return cudaErrorInvalidValue;
  switch (lg(pl.N1)) {
    case 8: return noise_ln<8>(a, pl, nfields, s);
    case 9: return noise_ln<9>(a, pl, nfields, s);
    case 10: return noise_ln<10>(a, pl, nfields, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_plane3_c2r(const PlaneArgs& pl, int64_t nfields, cudaStream_t s) {
  if (pl.R < 1 || pl.Q * pl.R != pl.N2 || pl.S3 != pl.M + 2 || nfields < 1 || !pl.status) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(pl.ws) & 15) || (!pl.zout && (reinterpret_cast<uintptr_t>(pl.out) & 15)))
    return cudaErrorInvalidValue;
  if (nfields * pl.N1 * pl.R >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
  switch (lg(pl.Q)) {
    case 4: return c2r_dispatch_q<4>(lg(pl.M), pl, nfields, s);
    case 5: return c2r_dispatch_q<5>(lg(pl.M), pl, nfields, s);
    case 6: return c2r_dispatch_q<6>(lg(pl.M), pl, nfields, s);
    case 7: return c2r_dispatch_q<7>(lg(pl.M), pl, nfields, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace grf
