// c2r pass fed by bulk asynchronous copies (the Tensor Memory Accelerator).
//
// The last pass of the 2-D and 3-D paths (step "FFT^-1" of Algorithm 2 along
// the contiguous axis d) reads the half spectrum once and writes the field
// once: it is bound by HBM.  In the plain row kernel every thread loads its
// own entries and waits for them before the transform, so a CTA computes only
// after its loads land.  Here a persistent CTA owns two shared-memory slots.
// A group of C rows whose entries are contiguous in the workspace (tile T
// divides C) arrives in one slot through one `cp.async.bulk` copy, completed
// on that slot's mbarrier, while the CTA transforms the group in the other
// slot.  The copy engine, not the threads, then keeps the HBM reads in
// flight.
//
// The slot holds the group exactly as the workspace lays it out: entry k of
// row c of the group at hrow_base(c, M, logT) + k T, where the last column
// pass left Z[k] = (X[k] + conj X[M-k]) + i e^{2 pi i k/N} (X[k] - conj X[M-k])
// (k < M).  Once Z is in registers, the same slot is the exchange buffer of
// the M-point transform.
//
// Every wait on an mbarrier is bounded (iterations and elapsed time).  A wait
// that gives up stores GRF_ERR_TIMEOUT in the plan's status word, waits
// (bounded again) for the CTA's copies still in flight, and the CTA returns.
#include "grf.h"
#include "bodies.cuh"
#include "tma.cuh"

namespace grf {

using namespace tma;

template <int P>
__global__ void __launch_bounds__(kMaxThreads<P>, kMinBlocks<P>)
    row_c2r_tma_kernel(RowArgs a, int64_t ngroups, int slot_elems, int* status) {
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw);
  float2* slot0 = reinterpret_cast<float2*>(smraw + 128);
  const int nthr = blockDim.x;
  const int t = threadIdx.x;
  const int C = a.C;
  const int c = t & (C - 1);
  const int tau = t / C;
  const int M = a.M;
  const int N = 2 * M;
  const int TPT = M / P;
  const uint32_t bytes = (uint32_t)((int64_t)(M + 1) * C * sizeof(float2));
  const uint32_t bar0 = smem_addr(&bars[0]);
  const uint32_t s0 = smem_addr(slot0);
  const uint32_t slot_bytes = (uint32_t)slot_elems * sizeof(float2);
  // offset of Z[0] of row c in a slot, as in the workspace
  const int cb = (int)hrow_base(c, M, a.logT);

  const int64_t first = blockIdx.x;
  const int64_t stride = gridDim.x;
  if (t == 0) {
    mbar_init(bar0);
    mbar_init(bar0 + 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int b = 0; b < 2; ++b) {
      const int64_t grp = first + b * stride;
      if (grp < ngroups)
        bulk_load(s0 + b * slot_bytes, a.inH + hrow_base(grp * C, M, a.logT), bytes, bar0 + 8 * b);
    }
  }
  __syncthreads();

  int64_t i = 0;
  for (int64_t grp = first; grp < ngroups; grp += stride, ++i) {
    const int b = (int)(i & 1);
    float2* sm = slot0 + (size_t)b * slot_elems;
    const bool ok = mbar_wait(bar0 + 8 * b, (uint32_t)((i >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicExch(status, (int)GRF_ERR_TIMEOUT);
        // the copies this CTA issued and has not seen complete: this group's
        // and, if issued, the next one's
        mbar_wait(bar0 + 8 * b, (uint32_t)((i >> 1) & 1));
        if (grp + stride < ngroups) mbar_wait(bar0 + 8 * (b ^ 1), (uint32_t)(((i + 1) >> 1) & 1));
      }
      __syncthreads();
      return;
    }
    float2 v[P];
#pragma unroll
    for (int q = 0; q < P; ++q) v[q] = sm[cb + ((tau + TPT * q) << a.logT)];
    fft_core<P, +1>(v, sm, tau, c, C, M, a.logM, a.twM, a.tws, nthr);
    float2* o = reinterpret_cast<float2*>(a.outR + (grp * C + c) * N);
#pragma unroll
    for (int q = 0; q < P; ++q) o[tau + TPT * q] = v[q];
    // the slot is refilled by the async proxy after the generic proxy's last
    // use of it in this CTA
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0 && grp + 2 * stride < ngroups)
      bulk_load(s0 + b * slot_bytes, a.inH + hrow_base((grp + 2 * stride) * C, M, a.logT), bytes, bar0 + 8 * b);
  }
}

bool c2r_tma_ok(const RowArgs& a) {
  if (a.C < 2 || (a.C & (a.C - 1)) || a.T < 1 || a.C % a.T) return false;
  if (a.nrows <= 0 || a.nrows % a.C) return false;
  if (reinterpret_cast<uintptr_t>(a.inH) & 15) return false;
  const int64_t bytes = (int64_t)(a.M + 1) * a.C * sizeof(float2);
  if (bytes % 16 || bytes >= (1 << 20)) return false;  // the mbarrier's transaction count
  return 2 * c2r_tma_slot_bytes(a.M, a.C) + 128 <= 227 * 1024;
}

size_t c2r_tma_slot_bytes(int M, int C) {
  const size_t e = row_smem_bytes(M, C);
  return (e + 127) / 128 * 128;
}

template <int P>
static cudaError_t launch_tma_t(const RowArgs& a, int ctas_per_sm, int num_sms, int* status, cudaStream_t s) {
  const int threads = a.C * a.M / P;
  const size_t slot = c2r_tma_slot_bytes(a.M, a.C);
  const size_t smem = 128 + 2 * slot;
  auto k = row_c2r_tma_kernel<P>;
  cudaError_t e = prepare_kernel((const void*)k, threads, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
  const int64_t ngroups = a.nrows / a.C;
  int64_t ctas = (int64_t)occ * num_sms;
  if (ctas > ngroups) ctas = ngroups;
  k<<<(unsigned)ctas, threads, smem, s>>>(a, ngroups, (int)(slot / sizeof(float2)), status);
  return cudaGetLastError();
}

cudaError_t launch_row_c2r_tma(int P, const RowArgs& a, int ctas_per_sm, int num_sms, int* status,
                               cudaStream_t s) {
  if (!c2r_tma_ok(a) || num_sms < 1 || !status) return cudaErrorInvalidValue;
  switch (P) {
    case 4: return launch_tma_t<4>(a, ctas_per_sm, num_sms, status, s);
    case 8: return launch_tma_t<8>(a, ctas_per_sm, num_sms, status, s);
    case 16: return launch_tma_t<16>(a, ctas_per_sm, num_sms, status, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace grf
