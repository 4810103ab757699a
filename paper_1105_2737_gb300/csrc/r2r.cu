// Neumann and Dirichlet fields (the cosine / sine transform variant that §1
// and §3 mention): on the box [0, L_i] with N_i intervals per axis,
//   f_J = sum_K t_K a_K prod_i E(k_i, j_i),  J, K in prod{0..N_i},
// E = cos(pi k j / N) (Neumann) or sin(pi k j / N) (Dirichlet), a_K real
// normals, t_K from the spectral density on the mirrored box of edges 2 L_i.
//
// One kernel, one launch per axis, in place on the caller's output: a CTA
// takes 2C lines of one axis (N + 1 points each), packs lines 2c and 2c + 1
// into one complex sequence x_a + i x_b, extends it evenly (Neumann: z_n =
// z_{2N-n}) or oddly (Dirichlet: z_{2N-n} = -z_n, z_0 = z_N = 0) to length 2N,
// runs one inverse FFT of length 2N, and keeps outputs 0..N.  For real even
// (odd) data the transform is real (imaginary), so the two lines separate:
//   Neumann:   y = e_0 + (-1)^j e_N + 2 sum_{0<n<N} e_n cos(pi n j / N)  -> (Re, Im)
//   Dirichlet: y = 2 sum_{0<n<N} e_n sin(pi n j / N)                     -> (Im, -Re)
// The factor 2 on interior coefficients is the extension's, so the table
// holds t_K = sqrt(w_K S(p_K) / |2D|) / 2^(number of interior k_i).
// The first launch (the last axis, contiguous rows) draws a_K itself, with
// the flat index j of K: call j >> 2, counter (q_lo, q_hi, 2, 0), words 2t,
// 2t + 1 (t = (j & 3) >> 1), even j the cosine normal, odd j the sine normal.
// Each line is staged through shared memory between global memory and the
// FFT's register layout, so that global loads and stores are coalesced along
// whichever direction is contiguous: along the points of a row, or across
// neighbouring lines of a strided axis.

#include <cstdlib>

#include "r2r.cuh"

namespace grf {

namespace {

using r2r::kR2rThreads;
using r2r::launch_r2r_t;
using r2r::R2R_NOISE_ROWS;
using r2r::R2R_LOAD_ROWS;
using r2r::R2R_LOAD_STRIDED;

template <int P>
cudaError_t launch_r2r_p(int src, const R2rArgs& a, cudaStream_t s) {
  const bool dir = a.bc == 2;
  switch (src) {
    case R2R_NOISE_ROWS: return dir ? launch_r2r_t<P, R2R_NOISE_ROWS, 2>(a, s) : launch_r2r_t<P, R2R_NOISE_ROWS, 1>(a, s);
    case R2R_LOAD_ROWS: return dir ? launch_r2r_t<P, R2R_LOAD_ROWS, 2>(a, s) : launch_r2r_t<P, R2R_LOAD_ROWS, 1>(a, s);
    default: return dir ? launch_r2r_t<P, R2R_LOAD_STRIDED, 2>(a, s) : launch_r2r_t<P, R2R_LOAD_STRIDED, 1>(a, s);
  }
}

}  // namespace

// FFT scratch (which also holds the tile), then per line: the offset of point
// 0, and for the noise launch its flat index in the field and its Philox key
size_t r2r_smem_bytes(int N, int C) { return (size_t)spad_h(2 * N) * C * sizeof(float2) + 3 * 2 * C * sizeof(int64_t); }

int r2r_points_per_thread(int N) { return 2 * N >= 16 ? 16 : 2 * N; }

int r2r_lines_per_cta(int N) {
  const int TPT = 2 * N / r2r_points_per_thread(N);
  int C = kR2rThreads / TPT;
  if (C > 256) C = 256;
  return C < 1 ? 1 : C;
}

cudaError_t launch_r2r(const R2rArgs& a, cudaStream_t s) {
  if (a.N < 2 || (a.N & (a.N - 1)) || a.N > 4096 || a.C < 1 || (a.C & (a.C - 1))) return cudaErrorInvalidValue;
  if (a.C * (2 * a.N / r2r_points_per_thread(a.N)) > kR2rThreads) return cudaErrorInvalidValue;
  if (a.noise && a.inner != 1) return cudaErrorInvalidValue;
  const int src = a.noise ? R2R_NOISE_ROWS : (a.inner == 1 ? R2R_LOAD_ROWS : R2R_LOAD_STRIDED);
  if (std::getenv("GRF_R2R_GENERAL") == nullptr) {  // "GRF_R2R_GENERAL": the run-time-geometry kernel only
    cudaError_t err = cudaSuccess;
    if (launch_r2r_spec(src, a, s, &err)) return err;
  }
  switch (r2r_points_per_thread(a.N)) {
    case 4: return launch_r2r_p<4>(src, a, s);
    case 8: return launch_r2r_p<8>(src, a, s);
    case 16: return launch_r2r_p<16>(src, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace grf
