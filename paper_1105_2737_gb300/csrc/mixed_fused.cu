// Fused passes of FP32 2-D plans whose sizes are 2^a 3^b 5^c 7^d (Algorithm
// 2): the same two passes as the power-of-two path, with the mixed-radix
// Stockham stages of mixed_fused.cuh run in shared memory.
//   pass 1: a CTA takes C1 columns kd of the half spectrum: draws the noise of
//           their N1 entries (rows k1 and k1 + N1/2 share a Philox call; the
//           planes kd in {0, M} take the conjugation rule), scales by s_K,
//           runs the inverse DFT of length N1 and writes X to the workspace
//           [j1 / T][kd][j1 % T];
//   pass 2: a CTA takes one tile of T rows j1: reads its (M + 1) T entries
//           (one contiguous run), forms the c2r split
//           Z[k] = (X[k] + conj X[M-k]) + i e^{2 pi i k / N2} (X[k] - conj X[M-k]),
//           runs the inverse DFT of length M and writes the N2 reals of each row.
#include "mixed_fused.cuh"
#include "bodies.cuh"

namespace grf {

namespace {

constexpr int kMixedThreads = 256;

__global__ void __launch_bounds__(kMixedThreads) mixed_noise_kernel(MixedArgs a) {
  extern __shared__ float2 sm[];
  const int N1 = a.N1, M = a.M, H = N1 / 2, C = a.C1;
  float2* bufA = sm;
  float2* bufB = sm + C * N1;
  const HalfGeom& g = a.g;
  const int64_t field = blockIdx.z;
  const uint64_t key = field_key(g, field);
  const float* stab = field_stab(g, field);
  const int kd0 = blockIdx.x * C;
  const int t = threadIdx.x, nthr = blockDim.x;
  const float r2 = 0.70710678118654752440f;
  const float rH = __frcp_rn((float)H);
  // noise x s_K into bufA[c N1 + k1]
  for (int idx = t; idx < C * H; idx += nthr) {
    const int c = C == 1 ? 0 : qdiv(idx, rH);
    const int i = idx - c * H;
    const int kd = kd0 + c;
    float2 x0 = make_float2(0.f, 0.f), x1 = make_float2(0.f, 0.f);
    if (kd <= M) {
      const float* srow = stab + (size_t)kd * (H + 1);
      const float s0 = __ldg(srow + i), s1 = __ldg(srow + (H - i));  // folded |k1|: i and N1 - (i + H)
      if (kd != 0 && kd != M) {  // rows i and i + H share one call
        const u32x4 w = philox_call((uint64_t)i * (uint64_t)(M + 1) + (uint64_t)kd, 0u, key);
        x0 = cscale(box_muller(w.x, w.y, g.trig), s0 * r2);
        x1 = cscale(box_muller(w.z, w.w, g.trig), s1 * r2);
      } else {
        x0 = cscale(alg2_xi_grid(i, 0, kd, N1, 1, M, key, g.trig), s0);
        x1 = cscale(alg2_xi_grid(i + H, 0, kd, N1, 1, M, key, g.trig), s1);
      }
    }
    bufA[c * N1 + i] = x0;
    bufA[c * N1 + i + H] = x1;
  }
  const float2* X = mixed_transform(bufA, bufB, N1, N1, C, a.rad1, a.nst1, a.st1);
  // X to the workspace tile layout, (j1 mod T) fastest, then the column
  const int logT = a.logT, T = 1 << logT;
  float2* ws = a.ws + field * a.ws_stride;
  const int64_t ncols = M + 1;
  const float rC = __frcp_rn((float)C);
  for (int idx = t; idx < C * N1; idx += nthr) {
    const int r = idx & (T - 1);
    const int rest = idx >> logT;
    const int jt = C == 1 ? rest : qdiv(rest, rC);
    const int c = rest - jt * C;
    const int kd = kd0 + c;
    if (kd > M) continue;
    ws[((int64_t)jt * ncols + kd) * T + r] = X[c * N1 + jt * T + r];
  }
}

__global__ void __launch_bounds__(512) mixed_c2r_kernel(MixedArgs a) {
  extern __shared__ float2 sm[];
  const int M = a.M, logT = a.logT, T = 1 << logT;
  const int ncols = M + 1;
  float2* bufA = sm;                // T x (M + 1): X, then a stage buffer
  float2* bufB = sm + T * (M + 1);  // T x M
  const int64_t field = blockIdx.z;
  const int jt = blockIdx.x;
  const int t = threadIdx.x, nthr = blockDim.x;
  const float2* ws = a.ws + field * a.ws_stride + (int64_t)jt * ncols * T;
  // the tile's contiguous run [kd][r] -> bufA[r (M + 1) + kd], eight loads in
  // flight per thread before they go to shared memory
  constexpr int U = 8;
  const int n = ncols * T;
  for (int i0 = t; i0 < n; i0 += U * nthr) {
    float2 x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = i0 + u * nthr;
      if (idx < n) x[u] = __ldcg(ws + idx);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = i0 + u * nthr;
      if (idx < n) bufA[(idx & (T - 1)) * ncols + (idx >> logT)] = x[u];
    }
  }
  __syncthreads();
  // Z of the c2r split -> bufB[r M + k]
  const float rM = __frcp_rn((float)M);
  for (int idx = t; idx < M * T; idx += nthr) {
    const int r = T == 1 ? 0 : qdiv(idx, rM);
    const int k = idx - r * M;
    const float2* x = bufA + r * ncols;
    bufB[idx] = c2r_pre(x[k], x[M - k], __ldg(a.tw2 + k));
  }
  // the M-point inverse DFT
  const float2* z = mixed_transform(bufB, bufA, M, M, T, a.rad2, a.nst2, a.st2);
  // f[2m] + i f[2m + 1] = z[m]: the tile's T rows are consecutive in the field
  const int64_t j1 = (int64_t)jt * T;
  float* rows = a.zout ? a.zout[field] + j1 * (2 * M) : a.out + (field * a.N1 + j1) * (2 * M);
  float2* o = reinterpret_cast<float2*>(rows);
  for (int idx = t; idx < M * T; idx += nthr) o[idx] = z[idx];
}

// tab[Ns - 1 + (r - 1) Ns + m] = e^{2 pi i m r / (R Ns)}, m < Ns, 1 <= r < R, of one stage
__global__ void mixed_stage_table_kernel(float2* tab, int R, int Ns) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (R - 1) * Ns) return;
  const int r = k / Ns + 1, m = k % Ns;
  double sn, cs;
  sincospi(2.0 * (double)(m * r) / (double)(R * Ns), &sn, &cs);
  tab[Ns - 1 + k] = make_float2((float)cs, (float)sn);
}

}  // namespace

cudaError_t build_mixed_stage_table(float2* tab, const int* radix, int nst, cudaStream_t s) {
  int Ns = 1;
  for (int st = 0; st < nst; ++st) {
    const int R = radix[st], cnt = (R - 1) * Ns;
    mixed_stage_table_kernel<<<(cnt + 255) / 256, 256, 0, s>>>(tab, R, Ns);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    Ns *= R;
  }
  return cudaSuccess;
}

size_t mixed_noise_smem_bytes(int N1, int C1) { return (size_t)2 * C1 * N1 * sizeof(float2); }
size_t mixed_c2r_smem_bytes(int M, int T) { return (size_t)T * (2 * M + 1) * sizeof(float2); }

cudaError_t launch_mixed_noise(const MixedArgs& a, int64_t nfields, cudaStream_t s) {
  if (a.C1 < 1 || a.logT < 0 || a.logT > 3 || a.nst1 < 1 || a.nst1 > 16 || nfields < 1 || nfields > 65535 ||
      a.N1 % (1 << a.logT))
    return cudaErrorInvalidValue;
  const size_t smem = mixed_noise_smem_bytes(a.N1, a.C1);
  cudaError_t e = prepare_kernel((const void*)mixed_noise_kernel, kMixedThreads, smem);
  if (e != cudaSuccess) return e;
  mixed_noise_kernel<<<dim3((unsigned)((a.M + 1 + a.C1 - 1) / a.C1), 1, (unsigned)nfields), kMixedThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mixed_c2r(const MixedArgs& a, int64_t nfields, cudaStream_t s) {
  if (a.logT < 0 || a.logT > 3 || a.nst2 < 1 || a.nst2 > 16 || nfields < 1 || nfields > 65535 ||
      a.N1 % (1 << a.logT) || (a.threads2 != 256 && a.threads2 != 512))
    return cudaErrorInvalidValue;
  const size_t smem = mixed_c2r_smem_bytes(a.M, 1 << a.logT);
  cudaError_t e = prepare_kernel((const void*)mixed_c2r_kernel, a.threads2, smem);
  if (e != cudaSuccess) return e;
  mixed_c2r_kernel<<<dim3((unsigned)(a.N1 >> a.logT), 1, (unsigned)nfields), a.threads2, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace grf
