/*
 * grf.h - C ABI of a GB300 (sm_103a) library that samples centered stationary
 * Gaussian random fields on periodic rectangular grids in 1, 2 and 3
 * dimensions by the FFT method of Lang & Potthoff, "Fast simulation of
 * Gaussian random fields" (arXiv 1105.2737).
 *
 * Method (paper section in brackets).  For a grid of N_1 x ... x N_d points
 * (every N_i even, §2) on a box with edge lengths L_1..L_d and a spectral
 * density S (the Lebesgue density gamma of the Bochner representation, §2):
 *   1. noise: independent normals arranged directly as Hermitian-symmetric
 *      Fourier coefficients xi_K on the half spectrum
 *      H = N_1 x ... x N_{d-1} x (N_d/2 + 1)  [§2 Lemma 1, Eq. conj; §3 Alg. 2],
 *      or, in the selectable mode of §3 Alg. 1, real normals z_j transformed by
 *      a forward DFT;
 *   2. scaling by s_K = sqrt(S(p_K)/|D|), |D| = L_1 ... L_d  [§2 Eq. drf, rules a)-e)];
 *   3. one inverse real-output FFT: f_j = sum_K s_K xi_K exp(+2 pi i K.j/N).
 * Readings fixed by this library where the paper leaves a choice:
 *   - p_K = (k~_i / L_i)_i with k~_i = k_i if k_i <= N_i/2 else k_i - N_i;
 *   - E|A_K|^2 = S(p_K)/|D| with an unnormalised inverse DFT, so that the
 *     variance is (1/|D|) sum_K S(p_K) (about sigma^2);
 *   - on the planes k_d in {0, N_d/2} a conjugate pair takes its value from
 *     the member with the larger row-major index in H;
 *   - noise is Philox4x32-10 (Salmon et al., SC'11) keyed by seed + b for
 *     field b, mapped to an exact uniform u = (2 (x >> 9) + 1) 2^-24 and to
 *     normals by Box-Muller; Algorithm 2, counter (q_lo, q_hi, 0, 0): in 1-D
 *     entry k_d uses call k_d >> 1, words 2 (k_d & 1) and 2 (k_d & 1) + 1; in
 *     2-D/3-D entry (k_1, k_mid, k_d) (k_mid = k_2 in 3-D, else 0) uses, with
 *     H = N_1/2, call ((k_1 mod H) N_mid + k_mid)(N_d/2 + 1) + k_d, words
 *     2 [k_1 >= H] and 2 [k_1 >= H] + 1 (N_mid = N_2 in 3-D, else 1); Algorithm 1 point j uses call
 *     j >> 2, counter (q_lo, q_hi, 1, 0), words 2t, 2t+1 with t = (j & 3) >> 1,
 *     even j taking the cosine normal and odd j the sine normal.
 *
 * Conventions for every call:
 *   - All arrays are C order (row-major, last axis contiguous).
 *   - A field is N_1 x ... x N_d real values, FP32 (float) or FP64 (double)
 *     according to the plan's precision.  A batch is `batch` fields back to
 *     back.
 *   - Pointers marked "device" are CUDA device (or managed) memory owned by the
 *     caller; the library never frees them.  The plan owns its tables and
 *     workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous and ordered on that stream.  A plan
 *     may be used by one stream at a time.
 *   - No C++ exception crosses this boundary.  Every call returns a status;
 *     argument errors are detected on the host before anything is launched.
 *     Errors raised by kernels (a bounded wait that ran out) are recorded in
 *     a device status word read by grf_status_word().
 */
#ifndef GRF_H_
#define GRF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GRF_OK = 0,
  GRF_ERR_INVALID_ARG = 1,   /* bad dimension, odd N_i, non-positive L_i or parameter, NULL pointer */
  GRF_ERR_UNSUPPORTED = 2,   /* valid for the method but not built (e.g. a prime factor of N_i above 7) */
  GRF_ERR_OOM = 3,           /* device allocation failed */
  GRF_ERR_CUDA = 4,          /* a CUDA runtime call failed */
  GRF_ERR_TIMEOUT = 5,       /* a bounded device wait ran out (persistent batch kernel) */
  GRF_ERR_NOT_HERMITIAN = 6  /* reserved: input half spectrum violates Eq. conj */
} grf_status;

typedef enum {
  GRF_MATERN = 0,     /* S = sigma^2 c (1 + ell^2 |2 pi p|^2)^(-nu-d/2),
                         c = (2 sqrt(pi) ell)^d Gamma(nu+d/2)/Gamma(nu): int S = sigma^2 */
  GRF_GAUSSIAN = 1,   /* S = sigma^2 (2 pi ell^2)^(d/2) exp(-2 pi^2 ell^2 |p|^2) */
  GRF_PAPER_POLY = 2  /* §4: S = sigma^2 (m^(k l) + (sum_i p_i^(2k))^l)^(-n) */
} grf_family;

typedef enum {
  GRF_ALG_TWO_FFT = 1, /* §3 Algorithm 1: real noise -> FFT -> scale -> inverse FFT */
  GRF_ALG_ONE_FFT = 2  /* §3 Algorithm 2 (default): Hermitian noise -> scale -> inverse FFT */
} grf_algorithm;

typedef enum {
  GRF_FP32 = 0, /* fused FP32 kernels; tables built in FP64 and rounded */
  GRF_FP64 = 1  /* plain FP64 form: one field per launch sequence, unfused */
} grf_precision;

typedef struct {
  int family;            /* grf_family */
  double sigma, ell, nu; /* Matern / Gaussian parameters (nu unused for Gaussian) */
  double m;              /* GRF_PAPER_POLY: mass parameter m > 0 */
  int k, l, n;           /* GRF_PAPER_POLY: positive integers */
  int normalize_discrete;/* 0: continuum normalisation (default);
                            1: rescale S so that (1/|D|) sum_K S(p_K) = sigma^2 exactly */
} grf_spectrum;

typedef enum {
  GRF_BC_NEUMANN = 1,  /* cosine transform: the field's mirror image across every face is smooth */
  GRF_BC_DIRICHLET = 2 /* sine transform: the field vanishes on every face */
} grf_boundary;

typedef struct grf_plan_s* grf_plan;

/*
 * grf_plan_create - validate a problem and build its tables (§3, inputs of
 * Algorithms 1 and 2: the box D with edges L_i, even N_i, the symmetric
 * positive gamma^(1/2), a Gaussian generator).
 *   out       : receives the plan handle (host pointer, must not be NULL).
 *   d         : dimension, 1..3.
 *   n         : host array of d grid sizes, each even, in [2, 4096] for axes
 *               1..d-1 and in [2, 8192] for axis d of a 2-D or 3-D grid; a 1-D
 *               grid goes up to 2^22 (Algorithm 2 in FP32 by a four-step c2r,
 *               and the FP64 plain form), 8192 for Algorithm 1 in FP32.  Every
 *               even 2^a 3^b 5^c 7^e is taken: FP32 plans on powers of two run
 *               the fused kernels; FP32 2-D Algorithm 2 plans with another
 *               size on some axis run two fused passes over the whole batch
 *               (noise + axis-1 DFT, then c2r rows; radix-2, 3, 4, 5, 7 and 8
 *               stages in shared memory); FP64 plans and the other FP32 plans
 *               off powers of two run the plain form (one launch sequence per
 *               field, radix-2, 3, 5 and 7 Stockham stages).  FP32 plans off
 *               powers of two have no adjoint, rfft or tuner.
 *   L         : host array of d edge lengths, each > 0.
 *   spec      : host pointer to the spectral density parameters.
 *   alg       : grf_algorithm.
 *   prec      : grf_precision.
 *   max_batch : largest batch later passed to grf_sample / grf_backward (>= 1);
 *               sizes the workspace.
 * Builds, on the current CUDA device, the FP64-computed and FP32-rounded
 * table of s_K on the folded half spectrum (S depends on |p_i| only), the
 * twiddle tables and the workspace.  Returns GRF_ERR_INVALID_ARG /
 * GRF_ERR_UNSUPPORTED / GRF_ERR_OOM / GRF_ERR_CUDA without leaking.
 */
grf_status grf_plan_create(grf_plan* out, int d, const int64_t* n, const double* L,
                           const grf_spectrum* spec, int alg, int prec, int64_t max_batch);

/*
 * grf_bc_plan_create - plan for fields with Neumann or Dirichlet boundary
 * conditions: the variant that §1 and §3 mention, in which the FFT is replaced
 * by the fast cosine or sine transform (the paper gives no formulas; this is
 * the library's reading).  The box [0, L_1] x ... x [0, L_d] carries N_i
 * intervals per axis, i.e. the points x_j = j L_i / N_i, j = 0..N_i, and a
 * field is the (N_1 + 1) x ... x (N_d + 1) array (C order, FP32)
 *   f_J = sum_K c_K a_K prod_i E(k_i, j_i),   J, K in prod{0..N_i},
 *   E = cos(pi k j / N_i) (GRF_BC_NEUMANN) or sin(pi k j / N_i) (GRF_BC_DIRICHLET),
 *   c_K = sqrt(w_K S(p_K) / |2D|),  p_K = (k_i / (2 L_i))_i,  |2D| = prod 2 L_i,
 *   w_K = prod_i w(k_i): Neumann w = 1 for k in {0, N_i}, 2 otherwise;
 *   Dirichlet w = 0 for k in {0, N_i}, 2 otherwise,
 * a_K independent N(0, 1): with the flat row-major index j of K, Philox call
 * j >> 2 with counter (q_lo, q_hi, 2, 0) and key seed + b, words 2t and 2t + 1
 * (t = (j & 3) >> 1), the Box-Muller cosine normal for even j and the sine
 * normal for odd j.  Its covariance is the method-of-images sum of the periodic
 * covariance c of the mirrored grid (2 N_i points, period 2 L_i):
 *   Cov(f_J, f_J') = 2^-d sum_{s in {+1,-1}^d} sgn(s) c(J + s J'),
 * sgn = 1 (Neumann) or prod_i (-s_i) (Dirichlet); a Dirichlet field is exactly
 * 0 on the faces.
 *   n    : host array of d interval counts, powers of two in [2, 4096].
 *   L    : host array of d edge lengths, each > 0.
 *   spec : any family; normalize_discrete must be 0 (else GRF_ERR_UNSUPPORTED).
 *   bc   : grf_boundary.
 * grf_sample on the plan writes batch * prod (N_i + 1) floats, grf_sample_host
 * the same fields to host memory; grf_plan_set_spectrum rebuilds c_K;
 * grf_cov_origin estimates the covariance of the corner with every point;
 * grf_plan_query answers keys 0 (points per field), 3..6 and 16 (bc);
 * grf_plan_timing records its launches (GRF_KERNEL_R2R_NOISE, GRF_KERNEL_R2R).
 * grf_backward, grf_rfft_forward and grf_plan_tune return an error for such
 * a plan.  The plan holds the FP64-computed, FP32-rounded c_K
 * (prod (N_i + 1) floats) and the twiddles.
 */
grf_status grf_bc_plan_create(grf_plan* out, int d, const int64_t* n, const double* L,
                              const grf_spectrum* spec, int bc, int64_t max_batch);

/*
 * grf_plan_set_spectrum - rebuild the plan's spectral tables for new
 * parameters of the same kind (§2 rule a): s_K and, for the adjoint, its
 * derivatives), on `stream`, without reallocating.  Used when the parameters
 * (sigma, ell, nu) change between calls, e.g. by a gradient step.
 *   spec : host pointer, validated as in grf_plan_create.
 * Later calls on the same stream see the new tables.
 */
grf_status grf_plan_set_spectrum(grf_plan p, const grf_spectrum* spec, void* stream);

/*
 * grf_plan_tune - choose the plan's schedules by timing them (no counterpart
 * in the paper): for each pass the radix (4, 8 or 16 points per thread), the
 * columns or rows per CTA, the row tile T of the 2-D workspace layout, and the
 * pipelining depth, by coordinate descent with CUDA events on `stream`.  The
 * winner is applied and stored in the tuning cache (GRF_TUNE_CACHE, default
 * $HOME/.cache/grf_gb300_tune.txt) under the GPU name, grid, algorithm and
 * max_batch; later grf_plan_create calls for the same key apply it, and
 * grf_plan_tune on such a plan keeps that schedule and returns GRF_OK without
 * timing (GRF_TUNE_FORCE=1 times again).  Setting GRF_TUNE=1 makes
 * grf_plan_create tune.  FP32 2-D and 3-D plans.  Allocates a temporary output
 * of at most 64 MiB (or one field) while it runs.
 */
grf_status grf_plan_tune(grf_plan p, void* stream);

/*
 * grf_sample - draw `batch` fields (§3 Algorithm 2, or Algorithm 1 if the plan
 * says so).  Field b uses Philox key seed + b.
 *   out : device pointer to batch * N_1 * ... * N_d floats (FP32 plan) or
 *         doubles (FP64 plan), C order, written completely.
 * 1 <= batch <= max_batch.
 */
grf_status grf_sample(grf_plan p, uint64_t seed, int64_t batch, void* out, void* stream);

/*
 * grf_sample_host - same fields as grf_sample, delivered to host memory.
 *   host_out : host pointer to batch fields.
 * Pinned host memory mapped into the device's address space is written by
 * the kernels directly.  Other host memory (or GRF_HOST_DIRECT=0): the device
 * computes into plan-owned buffers in chunks while earlier chunks are copied
 * out (each chunk over GRF_COPY_STREAMS copy streams, default 1), so copies
 * overlap compute.  Returns after the fields are in host memory
 * (synchronises `stream`).
 */
grf_status grf_sample_host(grf_plan p, uint64_t seed, int64_t batch, void* host_out, void* stream);

/*
 * grf_backward - adjoint of grf_sample with respect to the spectral parameters
 * (Algorithm 2 plans, FP32, Matern or Gaussian).  With f = IDFT(s xi) (§2 Eq. 2)
 * and an upstream gradient G = dLoss/df, per field b:
 *   dLoss/dtheta = sum_{K in H} w_K (d s_K / d theta) Re(xi_K conj(G^_K)),
 *   G^ = DFT(G) (exp(-2 pi i K.j/N)), w_K = 1 on the planes k_d in {0, N_d/2},
 *   2 elsewhere; xi is regenerated from the seed, never stored.
 *   grad_out    : device pointer to batch fields (same layout as grf_sample's out).
 *   grad_params : device pointer to batch * 3 doubles, written as
 *                 (dsigma, dell, dnu) per field (dnu = 0 for Gaussian).
 * The reduction over K is done in FP64.
 */
grf_status grf_backward(grf_plan p, uint64_t seed, int64_t batch, const void* grad_out,
                        double* grad_params, void* stream);

/*
 * grf_rfft_forward - forward real-to-complex DFT of `batch` real fields of the
 * plan's shape onto the half spectrum:
 *   out_halfspec[b, K] = sum_j in[b, j] exp(-2 pi i K.j/N),  K in H,
 * interleaved complex (re, im) of the plan's precision, C order over H.
 *   in, out_halfspec : device pointers.
 */
grf_status grf_rfft_forward(grf_plan p, int64_t batch, const void* in, void* out_halfspec,
                            void* stream);

/*
 * grf_batch_plan_create - plan for `count` independent fields of uneven shapes
 * and dimensions, each with its own Matern or Gaussian parameters (FP32,
 * Algorithm 2), sampled together (see grf_batch_set_mode for the two ways).
 *   d      : host array [count] of dimensions (1..3).
 *   n      : host array [count * 3]; field i uses n[3i .. 3i + d[i] - 1].
 *   L      : host array [count * 3], same indexing.
 *   spec   : host array [count] of spectra.
 *   prec   : must be GRF_FP32.
 * Schedules (transforms per tile, work order) are chosen by the built-in
 * tuner; the work queue and all tables live in plan-owned device memory.
 */
grf_status grf_batch_plan_create(grf_plan* out, int64_t count, const int* d, const int64_t* n,
                                 const double* L, const grf_spectrum* spec, int prec);

/*
 * grf_batch_sample - sample every field of a batch plan.  Field i uses
 * Philox key seed + i.
 *   out : host array [count] of device pointers, out[i] receiving field i
 *         (N_1 x ... x N_d floats).  The pointer array is copied at call time.
 * In the persistent mode, waits inside the kernel are bounded; if one runs
 * out the kernel records GRF_ERR_TIMEOUT in the plan's status word and returns.
 */
grf_status grf_batch_sample(grf_plan p, uint64_t seed, void* const* out, void* stream);

/*
 * grf_batch_graph_launch - the same as grf_batch_sample, replayed from a CUDA
 * graph captured for this (plan, mode, output pointer set).  In the per-shape
 * mode the call that captures the graph samples by direct launches and later
 * calls replay it; in the persistent mode the first call captures and replays.
 * The seed is read from plan memory at replay, so any seed may be used.
 */
grf_status grf_batch_graph_launch(grf_plan p, uint64_t seed, void* const* out, void* stream);

/*
 * grf_sample_2d_static - 2-D sampling that allocates no memory.  The paper has
 * no counterpart: this is a way of calling the sampler, not part of the method.
 *
 * For callers that cannot allocate device memory when they need a field: code
 * inside a host application that owns all of the device's memory (its own
 * pool, raw cudaMalloc not allowed), and latency-critical loops in which
 * cudaMalloc or cudaFree would implicitly synchronise the device.  It draws
 * the same fields as grf_sample on a plan created with
 * grf_plan_create(2, n, L, spec, GRF_ALG_ONE_FFT, GRF_FP32, ...): FP32,
 * Hermitian complex noise followed by one inverse FFT (the GRF_ALG_ONE_FFT
 * mode), field b with Philox key seed + b.
 *   n, L  : host arrays of 2 grid sizes (powers of two, 2 <= N_i <= 1024) and
 *           edge lengths (> 0); sizes above 1024 return GRF_ERR_INVALID_ARG.
 *   spec  : Matern, Gaussian or paper family; normalize_discrete is not
 *           supported here (GRF_ERR_UNSUPPORTED).
 *   out   : device pointer to batch * N_1 * N_2 floats, written completely.
 * Everything the call needs besides `out` (twiddles, the s_K table and one
 * field's half spectrum, at most 5.1 MiB) lives in a 6 MiB file-scope device
 * array that every device holds from the moment it loads this library until
 * the process exits.  The first call on a device looks up that array's device
 * address (once per device, with the device current), so make the first call
 * before any stream capture.  All calls on a device share the array and leave
 * their contents in it; each call rebuilds what it reads.  Calls that overlap
 * on the GPU race on the array: keep them on one stream at a time.
 */
grf_status grf_sample_2d_static(const int64_t* n, const double* L, const grf_spectrum* spec, uint64_t seed,
                                int64_t batch, float* out, void* stream);

/*
 * grf_batch_set_debug - test hook of a batch plan (no counterpart in the
 * paper).  withhold_field >= 0 makes the first pass of that field never report
 * completion, so the tiles that depend on it wait until their bounded wait
 * runs out: the launch then stops, returns, and grf_status_word reports
 * GRF_ERR_TIMEOUT.  timeout_ms > 0 sets the wait limit (default 2000 ms).
 * withhold_field = -1 restores normal operation.  Drops any captured graph.
 */
grf_status grf_batch_set_debug(grf_plan p, int withhold_field, double timeout_ms);

/*
 * grf_batch_set_mode - how a batch plan samples (no counterpart in the paper):
 *   0 (default): per-shape launches.  The fields are grouped by shape; each
 *     group is sampled by the plan kernels of that shape, one launch index per
 *     field (its Philox key, s_K table and output looked up by index), and the
 *     groups run on 8 streams forked from and joined back into `stream`.  No
 *     kernel waits on another.
 *   1: one persistent kernel over every (pass, tile) of every field, ordered by
 *     per-field pass counters with bounded waits.
 * Both draw the same fields (equal up to FP32 rounding).  A field withheld by
 * grf_batch_set_debug makes the plan run in mode 1 until it is released.
 * GRF_ERR_INVALID_ARG for another mode or a plan that is not a batch plan.
 */
grf_status grf_batch_set_mode(grf_plan p, int mode);

/*
 * grf_status_word - synchronise `stream`, read and clear the plan's device
 * status word (GRF_OK or GRF_ERR_TIMEOUT).
 */
grf_status grf_status_word(grf_plan p, void* stream);

/*
 * grf_cov_origin - the Monte Carlo covariance estimator of the paper's
 * statistical tests (§4: the 1-D study, and the covariance of one grid point
 * with all others behind its 2-D figures): samples the fields seed, seed + 1,
 * ..., seed + count - 1 of an FP32 plan (periodic, or Neumann / Dirichlet; in
 * chunks of max_batch, exactly as grf_sample would) and adds
 *   sums[j] += sum_b f_b(x_0) f_b(x_j),   j over all points of a field (flat C order),
 * where x_0 is the first grid point (the origin, or the corner of a boundary
 * field); Cov(x_0, x_j) = sums[j] / count.  FP64 sums, added in a fixed order
 * (the result does not depend on scheduling).
 *   sums : device pointer, one double per point of a field, caller-owned (zero
 *          it before the first call; later calls keep adding).
 * The plan keeps one chunk of fields and its partial sums (allocated on the
 * first call).  GRF_ERR_UNSUPPORTED for a batch plan, an FP64 plan, or a field
 * of more than 2^31 - 1 points.
 */
grf_status grf_cov_origin(grf_plan p, uint64_t seed, int64_t count, double* sums, void* stream);

/*
 * grf_philox_words - the raw generator behind R() of §3 Algorithms 1 and 2:
 * Philox4x32-10 words of calls q0 .. q0 + count - 1 with counter
 * (q_lo, q_hi, tag, 0) and key (lo, hi) of `key`, written as 4 uint32 per call
 * to the device array `out_words` (4 * count entries).  Exposed so that the
 * generator can be checked bit for bit against an independent implementation.
 */
grf_status grf_philox_words(uint64_t key, uint32_t tag, uint64_t q0, int64_t count, uint32_t* out_words,
                            void* stream);

/*
 * grf_alu_peak - measured lane-operation rate of the current device, the
 * denominator of the ALU view of the noise pass's roofline (no counterpart in
 * the paper).  Launches one short microbenchmark (eight independent chains
 * per thread, 8 CTAs of 256 threads per SM, tens of ms) on `stream`, times it
 * with CUDA events and writes operations per second to *ops_per_s (host).
 *   kind 0: FP32 fused multiply-adds (one operation each): the issue ceiling;
 *   kind 1: Philox4x32 rounds, counted as two 32 x 32 -> 64-bit multiplies,
 *           two three-input XORs and the round's two key additions shared by
 *           eight chains;
 *   kind 2: log2 and reciprocal square root (the special functions of
 *           Box-Muller), one operation each.
 * Allocates and frees a small device buffer; synchronises the stream.
 * GRF_ERR_INVALID_ARG for another kind or a NULL pointer.
 */
grf_status grf_alu_peak(int kind, double* ops_per_s, void* stream);

/*
 * Per-launch timing of a plan's kernels, for measurement (no counterpart in
 * the paper).  grf_plan_timing(p, cap) makes the next calls of grf_sample /
 * grf_backward / grf_rfft_forward on p bracket each of their kernel launches
 * with CUDA events on the launching stream, for at most `cap` launches
 * (cap = 0 switches it off).  grf_plan_timing_read() synchronises those
 * events and copies, for each recorded launch in order, its kernel kind
 * (GRF_KERNEL_*) and its duration in milliseconds into the host arrays
 * kinds[cap_out] and ms[cap_out]; it returns the number of launches recorded
 * (possibly more than cap_out) and starts a new recording.
 */
enum {
  GRF_KERNEL_NOISE_COLUMNS = 0, /* noise + Hermitian arrangement + s_K + inverse FFT along axis 1 */
  GRF_KERNEL_COLUMNS = 1,       /* complex FFT along a strided axis (axis 2, Alg. 1, adjoint) */
  GRF_KERNEL_ROWS_C2R = 2,      /* c2r along the last axis */
  GRF_KERNEL_ROWS_R2C = 3,      /* r2c along the last axis */
  GRF_KERNEL_ROWS_1D = 4,       /* 1-D single-pass kernels */
  GRF_KERNEL_PLAIN64 = 5,       /* one field of the plain form (a launch sequence; FP64, or FP32 off powers of two) */
  GRF_KERNEL_REDUCE = 6,        /* adjoint final sum */
  GRF_KERNEL_R2R_NOISE = 7,     /* boundary fields: noise + cosine / sine transform along the last axis */
  GRF_KERNEL_R2R = 8            /* boundary fields: cosine / sine transform along a strided axis */
};
grf_status grf_plan_timing(grf_plan p, int64_t cap);
int64_t grf_plan_timing_read(grf_plan p, int* kinds, float* ms, int64_t cap_out);

/* grf_plan_query - sizes: 0 = points per field (batch plans: total points),
 * 1 = half-spectrum entries per field, 2 = workspace bytes, 3 = dimension d,
 * 4..6 = N_1..N_3, 7 = tile T, 8/9 = radix and columns per CTA of the axis-1
 * pass, 10/11 = the same for the c2r pass, 12 = pipelining depth, 13/14 = the
 * axis-2 pass (3-D), 15 = 1 if the c2r pass is the persistent kernel fed by
 * bulk asynchronous copies (else the plain row kernel), 16 = the boundary
 * condition of a grf_bc_plan_create plan.  Returns -1 for an unknown key or a
 * NULL plan. */
int64_t grf_plan_query(grf_plan p, int key);

/* grf_plan_destroy - free the plan and everything it owns (NULL is allowed). */
grf_status grf_plan_destroy(grf_plan p);

/* grf_status_string - static text for a status code. */
const char* grf_status_string(grf_status s);

/* grf_last_error - static text describing the most recent error on this host
 * thread (empty if none). */
const char* grf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GRF_H_ */
