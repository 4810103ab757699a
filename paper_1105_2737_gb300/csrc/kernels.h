// Launch descriptors shared by the host planner and the FP32 FFT kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace grf {

// Sources and modes of the column pass (complex FFT along a strided axis).
enum ColSrc { COL_NOISE = 0, COL_LOAD = 1 };
enum ColMode {
  COL_INV = 0,            // inverse transform, store
  COL_FWD = 1,            // forward transform, store
  COL_FWD_SCALE_INV = 2,  // forward, multiply by s_K / sqrt(N_tot), inverse, store (Alg. 1)
  COL_FWD_ADJ = 3         // forward, then reduce against regenerated xi (adjoint)
};


// Sources and modes of the row pass (the contiguous last axis).
//   ROW_LOAD_Z: Z[k] = (X[k] + conj X[M-k]) + i e^{2 pi i k/N} (X[k] - conj X[M-k]),
//   k < M, as the last column pass leaves it (pair mode) in the half-spectrum
//   layout; ROW_NOISE_H: X drawn in the row (1-D).
enum RowSrc { ROW_LOAD_Z = 0, ROW_NOISE_H = 1, ROW_LOAD_REAL = 2, ROW_NOISE_REAL = 3 };
enum RowMode {
  ROW_C2R = 0,            // half spectrum (M+1) -> N = 2M reals: z = IFFT_M(Z), f[2m] + i f[2m+1] = z[m]
  ROW_R2C = 1,            // N reals -> half spectrum (M+1), forward
  ROW_R2C_SCALE_C2R = 2,  // 1-D Algorithm 1 in one pass
  ROW_R2C_ADJ = 3         // 1-D adjoint: forward r2c, then reduce against regenerated xi
};

// Geometry of the half spectrum H = N1 x Nmid x (M + 1) (d = 3), N1 x (M + 1)
// (d = 2, Nmid = 1) or (M + 1) (d = 1, N1 = Nmid = 1), and its noise keys.
struct HalfGeom {
  int d;
  int N1, Nmid, M;        // N_d = 2 M
  uint32_t Q;             // Philox calls per row: floor(M/2) + 1
  uint64_t seed;          // key of field b is seed + b (+ field0)
  int64_t field0;         // first field index of this launch
  const float* stab;      // s_K on the folded half spectrum, [kd][fmid][f1]: (M+1) x (Nmid/2+1) x (N1/2+1)
  const float* dstab;     // d s_K / d(ell), d s_K / d(nu) (2 tables, same shape), adjoint only
  float inv_sigma;        // d s_K / d sigma = s_K / sigma, adjoint only
  const float2* trig;     // exp(2 pi i h / 256), h < 256: coarse angles of Box-Muller
  float alg1_scale;       // 1 / sqrt(N_tot), Algorithm 1
  // Launches over fields of a batch plan (NULL / 0 otherwise): the batch index
  // of the field at launch index z (the key is seed + zfield[z]), the stride
  // between the fields' s_K tables, and the seed read from device memory (so
  // that a captured graph takes any seed).
  const int64_t* zfield;
  int64_t stab_zstride;
  const uint64_t* seed_ptr;
};

struct ColArgs {
  int N, logN;      // transform length along the axis
  int C;            // columns per CTA (blockDim.x = C * N / P)
  int64_t ncols;    // columns in a plane (consecutive in memory)
  int T, logT;      // row tile of the layout (1: plain [pos][col]; T: [pos/T][col][pos%T]), a power of 2
  int64_t ostride;  // element offset between planes (gridDim.y planes)
  int64_t bstride;  // element offset between fields (gridDim.z fields)
  const float2* in;
  float2* out;
  const float2* tw;   // tw[k] = exp(2 pi i k / N)
  const float2* tws;  // radix-16 stage tables (see fft_core)
  int plane_is_k1;   // COL_NOISE / scale / adjoint: the transform axis is axis 1
  int pitch3;        // 3-D noise pass of the plane path (T = 1): store (j1, k2, k3) at
                     // (j1 N2 + k2) pitch3 + k3 (rows padded to pitch3 = M + 2; 0: off)
  int zpair;         // COL_INV / COL_FWD_SCALE_INV on a plane of M+1 columns: slot p takes
                     // columns p and M - p and writes Z of the c2r split (see col_body)
  const float2* twz; // zpair: exp(2 pi i k / N_d), k <= M/2
  HalfGeom g;
  double* partial;   // COL_FWD_ADJ: 3 doubles per CTA, indexed by linear block id
};

struct RowArgs {
  int M, logM;        // complex FFT length; real length N = 2 M
  int C;              // rows per CTA (blockDim.x = C * M / P)
  int64_t nrows;      // rows in this launch (all fields)
  int64_t rows_per_field;
  int T, logT;        // tile of the half-spectrum layout (1: plain rows), a power of 2
  const float2* inH;  // ROW_LOAD_H
  const float* inR;   // ROW_LOAD_REAL
  float2* outH;       // ROW_R2C
  float* outR;        // ROW_C2R, ROW_R2C_SCALE_C2R
  const float2* twM;  // exp(2 pi i k / M), k < M
  const float2* twN;  // exp(2 pi i k / N), k < N
  const float2* tws;  // radix-16 stage tables (see fft_core)
  HalfGeom g;
  double* partial;    // ROW_R2C_ADJ
  float* const* zout; // batch plans: output of the field at launch index z (NULL: outR + z field size)
};

// Four-step c2r for long 1-D grids (Algorithm 2): M = N/2 = A * B.
//   stage 1: for every column k1 < A, the sequence Z[k1 + A k2] (k2 < B) of the
//            c2r split, built from X[k] = s_k xi_k and X[M - k] drawn in
//            registers, inverse FFT of length B, times exp(2 pi i n2 k1 / M);
//            stored as Y[k1 / T][n2][k1 % T] (T = columns per CTA of stage 1).
//   stage 2: for every n2 < B, inverse FFT of length A over k1 gives
//            z[n2 + B n1]; f[2m] = Re z[m], f[2m + 1] = Im z[m].
struct FourStepArgs {
  int A, logA, B, logB, M, N;
  int C;             // columns per CTA
  int T, logT;       // tile of Y (the column count per CTA of stage 1)
  float2* Y;         // one field = M complex, fields back to back
  const float2* Yin;
  float* out;        // N floats per field
  const float2* twA; // exp(2 pi i k / A)
  const float2* twB;
  const float2* twM; // exp(2 pi i k / M), k < M
  const float2* twN; // exp(2 pi i k / N), k < M
  const float2* tws;
  const float* stab; // s_k, k <= M
  const float2* trig;  // exp(2 pi i h / 256)
  uint64_t seed;
  int64_t field0;
  // batch plans (NULL / 0 otherwise), as in HalfGeom and RowArgs
  const int64_t* zfield;
  int64_t stab_zstride;
  const uint64_t* seed_ptr;
  float* const* zout;
  // s_k laid out along k2 for the paired first stage: stabT[k1 B + k2] =
  // s_{k1 + A k2} (M entries per field, stride stabT_zstride); s_M from stab
  const float* stabT;
  int64_t stabT_zstride;
  const float2* tw2B;  // exp(2 pi i j / (2 B)), j < 2B
  const float2* twMA;  // exp(2 pi i j / A) = exp(2 pi i j B / M), j < A
};
// stabT of a four-step plan from its s_k table (1 field).
cudaError_t build_stab_fourstep(float* stabT, const float* stab, int A, int B, cudaStream_t s);
// stage 1, 2, or 3 = stage 1 with mirror-closed column pairs (a.C / 2 pairs per
// CTA, Y tile a.T = a.C / 2; each X drawn once, see fourstep1_pair_body).
cudaError_t launch_fourstep(int stage, int P, const FourStepArgs& a, int64_t nfields, cudaStream_t s);
// The compiled geometries of stages 3 and 2 (fourstep_spec.cu): true if one
// matched and was launched (its status in *err).
bool launch_fourstep_spec(int stage, const FourStepArgs& a, int64_t nfields, cudaStream_t s, cudaError_t* err);

// One axis of a Neumann / Dirichlet field (r2r.cu): lines of N + 1 points
// (N a power of two in [2, 4096]) along an axis of the field array, lines
// (o, i) starting at o (N + 1) inner + i within a field; C complex sequences
// (2C lines) per CTA, C * 2N / points_per_thread <= 512 threads.
struct R2rArgs {
  float* f;                 // the batch of fields, transformed in place
  int64_t field_stride;     // points per field
  int64_t nlines;           // lines over the batch
  int64_t lines_per_field;
  int64_t inner;            // stride between the points of a line (1: contiguous rows)
  int N, logNF;             // intervals per line; log2 of the FFT length 2N
  int C, logC, logG;        // sequences per CTA, log2 C, log2 (2C)
  int bc;                   // 1: Neumann (cosine), 2: Dirichlet (sine)
  int d, axis;              // dimension and the axis of this launch
  int64_t pts[3];           // points per axis, N_i + 1
  int noise;                // 1: draw a_K t_K (contiguous rows only) instead of loading
  const float* tab;         // t_K, field layout (noise launch only)
  uint64_t seed;            // key of field b is seed + field0 + b
  int64_t field0;
  const float2* tw;         // exp(2 pi i k / 2N), k < 2N
  const float2* tws;        // radix-16 stage tables (see fft_core)
  const float2* trig;       // exp(2 pi i h / 256): coarse angles of Box-Muller
};
cudaError_t launch_r2r(const R2rArgs& a, cudaStream_t s);
size_t r2r_smem_bytes(int N, int C);
int r2r_points_per_thread(int N);
int r2r_lines_per_cta(int N);  // the default C for lines of N + 1 points

// The 3-D plane path of Algorithm 2 (plane3d.cu).  N2 = R Q.  Pass 1 draws the
// noise, runs the inverse FFT along axis 1 and the first radix-R step of the
// axis-2 inverse FFT (decimation in frequency), and writes R independent
// sub-planes per j1:
//   ws[field][j1][s][k'][k3] = w^{k' s} sum_r X[j1, k' + Q r, k3] e^{2 pi i r s / R},
//   w = e^{2 pi i / N2}, k' < Q, k3 <= M (row pitch S3 = M + 2);
// pass 2 takes one sub-plane per CTA (one bulk copy into shared memory), runs
// the length-Q inverse FFTs along k' (giving the axis-2 outputs j2 = s + R j'),
// forms the c2r split and the M-point inverse FFT of every row, and writes each
// row of N3 = 2M reals with one bulk copy.
struct PlaneArgs {
  int N1, N2, M;
  int R, Q, S3;
  float2* ws;          // sub-planes of this launch's fields
  float* out;          // fields [field][j1][j2][N3]
  const float2* tw;    // tw[L + k] = exp(2 pi i k / L)
  const float2* tws;   // stage tables (see fft_core)
  int* status;         // GRF_ERR_TIMEOUT if a bulk copy's wait ran out
  float* const* zout;  // batch plans: output of the field at launch index z (NULL: out)
};
// R for a 3-D plan (1, 2 or 4), or 0 if the plane path does not apply.  For
// N1 < 256 pass 1 is the ordinary noise + axis-1 column pass writing whole
// planes (R = 1) with rows padded to M + 2 (ColArgs::pitch3).
int plane3_radix(int N1, int N2, int M);
size_t plane3_ws_entries(int N1, int N2, int M);  // per field
cudaError_t launch_plane3_noise(const ColArgs& a, const PlaneArgs& pl, int64_t nfields, cudaStream_t s);
cudaError_t launch_plane3_c2r(const PlaneArgs& pl, int64_t nfields, cudaStream_t s);

// The fused passes of FP32 2-D plans of sizes 2^a 3^b 5^c 7^d (mixed_fused.cu),
// Algorithm 2: pass 1 (noise + the axis-1 inverse DFT of C1 columns per CTA,
// in shared memory) writes X to ws [j1 / T][kd][j1 % T]; pass 2 (one tile of
// T rows per CTA) forms the c2r split and the M-point inverse DFT.  Radix lists
// rad1 (length N1) and rad2 (length M) take radices 2, 3, 4, 5, 7, 8.
struct MixedArgs {
  int N1, M;
  int logT, C1;        // workspace tile T = 2^logT rows (T divides N1); columns per CTA of pass 1
  int threads2;        // threads per CTA of pass 2 (256 or 512)
  int nst1, nst2;
  int rad1[16], rad2[16];
  const float2* st1;   // stage tables of the lengths N1 and M (build_mixed_stage_table)
  const float2* st2;
  const float2* tw2;   // e^{2 pi i k / N2}, k < N2
  HalfGeom g;          // noise keys and the folded s_K table
  float2* ws;
  int64_t ws_stride;   // entries per field (N1 (M + 1))
  float* out;
  float* const* zout;  // batch plans: output of the field at launch index z (NULL: out)
};
// The stage table of a length N with radices radix[0..nst): N - 1 entries,
// stage s (span Ns) at Ns - 1: e^{2 pi i m r / (R Ns)} at (r - 1) Ns + m.
cudaError_t build_mixed_stage_table(float2* tab, const int* radix, int nst, cudaStream_t s);
size_t mixed_noise_smem_bytes(int N1, int C1);
size_t mixed_c2r_smem_bytes(int M, int T);
cudaError_t launch_mixed_noise(const MixedArgs& a, int64_t nfields, cudaStream_t s);
cudaError_t launch_mixed_c2r(const MixedArgs& a, int64_t nfields, cudaStream_t s);

// Host launchers (fft_kernels.cu).  P is the points per thread of the
// transform (16 if the length is >= 16, else the length itself).
cudaError_t launch_col(int src, int mode, int P, const ColArgs& a, dim3 grid, cudaStream_t s);
cudaError_t launch_row(int src, int mode, int P, const RowArgs& a, dim3 grid, cudaStream_t s);
// The noise + axis-1 pass (noise_kernels.cu), compiled per noise variant.
cudaError_t launch_col_noise(int P, const ColArgs& a, dim3 grid, cudaStream_t s);
// Compile-time-geometry forms (spec_*.cu): launch and return true if the
// launch has one, else return false and launch nothing.
bool launch_col_noise_spec(int P, const ColArgs& a, dim3 grid, cudaStream_t s, cudaError_t* err);
// The 2-D noise pair pass specialised for those geometries and the tile T
// (noise_fast.cu): launch and return true if the launch has that form.
bool launch_noise_pair_fast(int P, const ColArgs& a, dim3 grid, cudaStream_t s, cudaError_t* err);
bool launch_col_load_pair_spec(int P, const ColArgs& a, dim3 grid, cudaStream_t s, cudaError_t* err);
bool launch_row_c2r_spec(int P, const RowArgs& a, dim3 grid, cudaStream_t s, cudaError_t* err);
// Grid-stride forms (ctas CTAs walk all tiles) of the noise + axis-1 pass and the c2r pass.
cudaError_t launch_col_noise_gs(int P, const ColArgs& a, dim3 tiles, int ctas, cudaStream_t s);
cudaError_t launch_row_c2r_gs(int P, const RowArgs& a, int64_t ntiles, int ctas, cudaStream_t s);
size_t col_smem_bytes(int N, int C);
size_t col_pair_smem_bytes(int N, int C);  // pair mode (ColArgs::zpair)
// The c2r pass as a persistent kernel fed by bulk asynchronous copies
// (c2r_tma.cu): groups of C rows (C a power of two >= 2, the workspace tile T
// dividing C, nrows a multiple of C), two shared-memory slots per CTA.  At most
// ctas_per_sm CTAs per SM (0: as many as fit).  A wait that times out stores
// GRF_ERR_TIMEOUT in *status.
bool c2r_tma_ok(const RowArgs& a);
size_t c2r_tma_slot_bytes(int M, int C);
cudaError_t launch_row_c2r_tma(int P, const RowArgs& a, int ctas_per_sm, int num_sms, int* status, cudaStream_t s);
// The Monte Carlo covariance estimator of the 1-D study (study.cu): adds
// sum_b f[b][0] f[b][j] (b < B, j < N) onto sums[j] in FP64, through
// `partial` (cov_origin_partial_count(B) x N doubles).
int64_t cov_origin_partial_count(int64_t B);
cudaError_t launch_cov_origin(const float* f, int64_t B, int N, double* partial, double* sums, cudaStream_t s);
// Launch bounds of the transform kernels: 256 threads per CTA for radix 16
// (3 CTAs per SM), 512 for radix 8 (N = 4096 needs 512 threads of 8 points),
// 1024 for radix 4 and below.
template <int P>
constexpr int kMaxThreads = P >= 16 ? 256 : (P == 8 ? 512 : 1024);
template <int P>
constexpr int kMinBlocks = P >= 16 ? 3 : (P == 8 ? 2 : 1);
// Dynamic shared memory and the L1/shared carveout of a kernel for a launch shape.
cudaError_t prepare_kernel(const void* k, int threads, size_t smem);
size_t row_smem_bytes(int M, int C);
int points_per_thread(int n);

// Table kernels (tables.cu).  All arithmetic in FP64, stored rounded to FP32.
struct SpecParams {
  int family;
  double sigma, ell, nu, m;
  int k, l, n;
  double scale;       // multiplies S/|D| (discrete normalisation), normally 1
  double L[3];
  int nn[3];          // N_1..N_d
  int d;
};
// tw[L + k] = exp(2 pi i k / L) for powers of two L <= maxlen, then (at
// offset 2 maxlen) the stage tables: radix 16 (spans 16, 256), radix 8 (8, 64,
// 512), radix 4 (4, 16, 64, 256, 1024), (P - 1) Ns entries per span; then the
// tables of the final radix-2/4/8 stage of the radix-16 engine (spans 16 and
// 256, see small_stage_offset).
constexpr int kStageTableMain = 15 * (16 + 256) + 7 * (8 + 64 + 512) + 3 * (4 + 16 + 64 + 256 + 1024);
constexpr int kSmallStageEntries = (1 + 3 + 7) * (16 + 256);
constexpr int kStageTableEntries = kStageTableMain + kSmallStageEntries;
// Offset (within the stage tables) of the final radix-R stage (R in {2, 4, 8})
// after radix-16 stages of total span Ns (16 or 256): (R - 1) Ns entries,
// entry (r - 1) Ns + j = exp(+2 pi i j r / (R Ns)), j < Ns, r = 1..R-1.
__host__ __device__ constexpr int small_stage_offset(int R, int Ns) {
  return kStageTableMain + (Ns == 16 ? 0 : 11 * 16) + (R == 2 ? 0 : (R == 4 ? Ns : 4 * Ns));
}
cudaError_t build_twiddles(float2* tw, int maxlen, cudaStream_t s);
cudaError_t build_twiddles_d(double2* tw, int maxlen, cudaStream_t s);
cudaError_t build_stab(float* stab, float* dstab, const SpecParams& sp, double dig_a_minus_nu,
                       cudaStream_t s);
cudaError_t build_stab_d(double* stab, const SpecParams& sp, cudaStream_t s);
// t_K of a Neumann (bc = 1) / Dirichlet (bc = 2) field on prod{0..N_i} in
// field layout (last axis fastest): sqrt(S(p_K) / |2D|) with p_K = (k_i / (2 L_i))_i,
// times 1 (k_i in {0, N_i}, Neumann), 0 (k_i in {0, N_i}, Dirichlet) or
// 1/sqrt(2) (interior k_i) per axis.  sp.nn holds the intervals N_i.
cudaError_t build_bc_table(float* tab, const SpecParams& sp, int bc, cudaStream_t s);
cudaError_t philox_words(uint64_t key, uint32_t tag, uint64_t q0, int64_t count, uint32_t* out, cudaStream_t s);
cudaError_t reduce_partials(const double* partial, int64_t nblk_per_field, int64_t nfields,
                            double* out, cudaStream_t s);

}  // namespace grf
