"""Plain FP64 CPU oracle for the FFT method of Lang & Potthoff,
"Fast simulation of Gaussian random fields" (arXiv 1105.2737).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The
product path (the CUDA library and its Python binding) never calls it, and this
module shares no code with it: every step below is written out in numpy, FP64,
as the paper defines it, with no blocking, fusion or reordering.

What it computes, per field (paper section in brackets):

* frequencies p_K of the DFT grid, wrapped to [-N/2, N/2]            [§2 rule e)]
* the spectral density S(p) of the chosen family, and
  s_K = sqrt(S(p_K) / |D|)                                           [§2 Eq. drf]
* counter-based noise: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11)
  -> exact uniform in (0,1) -> Box-Muller                            [§3 Alg. 1/2, R()]
* Algorithm 2: the Hermitian arrangement of the noise on the half
  spectrum H (k_d = 0..N_d/2) and one inverse DFT                    [§2 Lemma 1, Eq. conj, §3 Alg. 2]
* Algorithm 1: real noise -> forward DFT -> scale -> inverse DFT     [§2 Eq. 1, §3 Alg. 1]
* exact covariance c(r) = (1/|D|) sum_K S(p_K) cos(2 pi K.r/N)      [§2, consequence of rules a)-d)]
* Neumann / Dirichlet fields by cosine / sine sums on the mirrored box,
  with the method-of-images covariance                              [§1, §3 remark on DCT/DST]
* the radially binned power-spectrum loss and its analytic gradient
  with respect to (sigma, ell, nu) (no counterpart in the paper; the
  field's derivative follows from Eq. 2).

Conventions (the readings of the paper that this oracle fixes):

* p_K has components k~_i / L_i with k~_i = k_i if k_i <= N_i/2 else k_i - N_i
  (cycles per unit length, the Bochner convention exp(-2 pi i (p, x)) of §2).
  The literal (k_i - N_i/2)/l_i of the algorithm remarks is the same set of
  points for an fft-shifted array; on an unshifted DFT array it would flip the
  sign of every other covariance lag.
* E|A_K|^2 = S(p_K)/|D| and the inverse DFT is unnormalised with exp(+2 pi i);
  then Var f = (1/|D|) sum_K S(p_K), a Riemann sum of int S = sigma^2, and
  Algorithms 1 and 2 have the same law (§2 Eq. 2).
* On the planes k_d in {0, N_d/2} the pair {K, -K} takes its value from the
  member with the larger row-major half-spectrum index: this is what survives
  the sequential loop of Algorithm 2, where the later iteration overwrites the
  conjugate partner written by the earlier one.
* Noise counters: field b of a call with seed s uses key (lo, hi) of s + b.
  Algorithm 2, counter (q_lo, q_hi, 0, 0), M = N_d/2:
    d = 1, entry k_d: call q = k_d >> 1, words 2(k_d & 1) and 2(k_d & 1) + 1;
    d >= 2, entry (k_1, k_mid, k_d) (k_mid = k_2 in 3-D, 0 in 2-D, N_mid = N_2
    or 1), H = N_1/2: call q = ((k_1 mod H) N_mid + k_mid)(M + 1) + k_d, words
    2 [k_1 >= H] and 2 [k_1 >= H] + 1 (rows k_1 and k_1 + H share a call).
  Algorithm 1, real grid point with
  flat index j: call q = j >> 2, counter (q_lo, q_hi, 1, 0), pair
  t = (j & 3) >> 1 uses words 2t, 2t+1; the even j takes the cosine normal,
  the odd j the sine normal.
* Uniform u = (2 (x >> 9) + 1) * 2^-24, exact in FP32 and FP64, in (0, 1).
  Box-Muller: rho = sqrt(-2 ln u_a), z_re = rho cos(2 pi u_b),
  z_im = rho sin(2 pi u_b), with u_a from the first word of the pair.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` (library routines, closed forms printed in the
paper, brute-force covariance, finite differences, an independent Philox).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

# ---------------------------------------------------------------------------
# Spectral families
# ---------------------------------------------------------------------------

MATERN = 0
GAUSSIAN = 1
PAPER_POLY = 2

ALG_TWO_FFT = 1  # Algorithm 1 (real noise -> FFT -> scale -> inverse FFT)
ALG_ONE_FFT = 2  # Algorithm 2 (Hermitian noise -> scale -> inverse FFT)

TAG_ALG2 = 0
TAG_ALG1 = 1


@dataclass
class Spectrum:
    """Parameters of the spectral density gamma of §2.

    family MATERN:   S(p) = sigma^2 c (1 + ell^2 |2 pi p|^2)^(-nu - d/2),
                     c = (2 sqrt(pi) ell)^d Gamma(nu + d/2) / Gamma(nu), so that
                     int S dp = sigma^2 (unit variance for sigma = 1).
    family GAUSSIAN: S(p) = sigma^2 (2 pi ell^2)^(d/2) exp(-2 pi^2 ell^2 |p|^2),
                     the transform of sigma^2 exp(-|r|^2 / (2 ell^2)).
    family PAPER_POLY (§4): S(p) = sigma^2 (m^(k l) + (sum_i p_i^(2k))^l)^(-n).
    normalize_discrete: rescale S so that (1/|D|) sum_K S(p_K) = sigma^2.
    """

    family: int = MATERN
    sigma: float = 1.0
    ell: float = 0.1
    nu: float = 1.5
    m: float = 1.0
    k: int = 1
    l: int = 1
    n: int = 1
    normalize_discrete: int = 0


def matern_constant(ell: float, nu: float, d: int) -> float:
    """c = (2 sqrt(pi) ell)^d Gamma(nu + d/2) / Gamma(nu).

    From int_{R^d} (1 + |u|^2)^(-a) du = pi^(d/2) Gamma(a - d/2) / Gamma(a)
    with u = 2 pi ell p and a = nu + d/2.
    """
    return (2.0 * math.sqrt(math.pi) * ell) ** d * math.exp(
        math.lgamma(nu + d / 2.0) - math.lgamma(nu))


def spectral_density(p: Sequence[np.ndarray], spec: Spectrum) -> np.ndarray:
    """S(p) for p given as a list of d coordinate arrays (cycles / unit length)."""
    d = len(p)
    p2 = sum(np.asarray(pi, dtype=np.float64) ** 2 for pi in p)
    if spec.family == MATERN:
        c = matern_constant(spec.ell, spec.nu, d)
        w2 = (2.0 * math.pi) ** 2 * p2
        return spec.sigma ** 2 * c * (1.0 + spec.ell ** 2 * w2) ** (-spec.nu - d / 2.0)
    if spec.family == GAUSSIAN:
        return (spec.sigma ** 2 * (2.0 * math.pi * spec.ell ** 2) ** (d / 2.0)
                * np.exp(-2.0 * math.pi ** 2 * spec.ell ** 2 * p2))
    if spec.family == PAPER_POLY:
        s2k = sum(np.asarray(pi, dtype=np.float64) ** (2 * spec.k) for pi in p)
        return spec.sigma ** 2 * (spec.m ** (spec.k * spec.l) + s2k ** spec.l) ** (-float(spec.n))
    raise ValueError("unknown spectral family")


def wrapped_index(k: np.ndarray, N: int) -> np.ndarray:
    """k~ = k if k <= N/2 else k - N (§2 rule e), read as DFT frequencies)."""
    k = np.asarray(k)
    return np.where(k <= N // 2, k, k - N)


def frequency_grid(n: Sequence[int], L: Sequence[float], half: bool = False):
    """Coordinate arrays p_i (broadcastable, 'ij' indexing) for the full grid
    K^N, or for the half spectrum H (last axis k_d = 0..N_d/2) if half."""
    d = len(n)
    axes = []
    for i in range(d):
        cnt = n[i] // 2 + 1 if (half and i == d - 1) else n[i]
        k = np.arange(cnt)
        axes.append(wrapped_index(k, n[i]).astype(np.float64) / L[i])
    return np.meshgrid(*axes, indexing="ij")


def discrete_normaliser(n, L, spec: Spectrum) -> float:
    """Factor applied to S when normalize_discrete is set: sigma^2 / ((1/|D|) sum_K S)."""
    vol = float(np.prod(L))
    S = spectral_density(frequency_grid(n, L), spec)
    return spec.sigma ** 2 / (S.sum() / vol)


def scaled_density(n, L, spec: Spectrum, half: bool = False) -> np.ndarray:
    """S(p_K)/|D| on the full grid or on H, including the optional discrete normalisation."""
    vol = float(np.prod(L))
    S = spectral_density(frequency_grid(n, L, half=half), spec) / vol
    if spec.normalize_discrete:
        S = S * discrete_normaliser(n, L, spec)
    return S


def sqrt_scale(n, L, spec: Spectrum, half: bool = False) -> np.ndarray:
    """s_K = sqrt(S(p_K)/|D|), the factor gamma(p_K)^(1/2) |A|^(-1) of Eq. drf."""
    return np.sqrt(scaled_density(n, L, spec, half=half))


# ---------------------------------------------------------------------------
# Philox4x32-10 and Box-Muller
# ---------------------------------------------------------------------------

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon et al., SC'11).

    ctr: 4 uint32 arrays (broadcastable); key: 2 uint32 arrays or ints.
    Each round: (hi0, lo0) = M0 * c0 and (hi1, lo1) = M1 * c2 as 64-bit
    products; the new counter is (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the
    key is then bumped by the Weyl constants (W0, W1).  Returns 4 uint32 arrays.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in ctr)
    k0 = np.asarray(key[0], dtype=np.uint64) & MASK32
    k1 = np.asarray(key[1], dtype=np.uint64) & MASK32
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = np.uint64(PHILOX_M0) * c0
        p1 = np.uint64(PHILOX_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return tuple(np.asarray(c, dtype=np.uint32) for c in (c0, c1, c2, c3))


def key_of(seed: int):
    """(lo, hi) 32-bit halves of a 64-bit key."""
    s = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (s & MASK32, s >> 32)


def uniform_from_word(x: np.ndarray) -> np.ndarray:
    """u = (2 (x >> 9) + 1) 2^-24: the 23 top bits of x, centred; exact in FP32."""
    x = np.asarray(x, dtype=np.uint64)
    return ((x >> np.uint64(9)) * np.uint64(2) + np.uint64(1)).astype(np.float64) * 2.0 ** -24


def box_muller(wa: np.ndarray, wb: np.ndarray):
    """Two independent N(0,1) from two words: rho = sqrt(-2 ln u_a), angle 2 pi u_b."""
    ua = uniform_from_word(wa)
    ub = uniform_from_word(wb)
    rho = np.sqrt(-2.0 * np.log(ua))
    return rho * np.cos(2.0 * math.pi * ub), rho * np.sin(2.0 * math.pi * ub)


def philox_words(q: np.ndarray, tag: int, seed: int):
    """The 4 Philox words of call q (uint64 array) with counter (q_lo, q_hi, tag, 0)."""
    q = np.asarray(q, dtype=np.uint64)
    ctr = (q & MASK32, q >> np.uint64(32), np.full(q.shape, tag, np.uint64), np.zeros(q.shape, np.uint64))
    return philox4x32_10(ctr, key_of(seed))


# ---------------------------------------------------------------------------
# Index sets of §2: self-conjugate points, conjugate partners, L^N
# ---------------------------------------------------------------------------

def half_shape(n: Sequence[int]):
    """Shape of the half spectrum H: N_1 x ... x N_{d-1} x (N_d/2 + 1)."""
    return tuple(n[:-1]) + (n[-1] // 2 + 1,)


def negate_index(K: Sequence[int], n: Sequence[int]):
    """-K mod N."""
    return tuple((-k) % N for k, N in zip(K, n))


def is_self_conjugate(K, n) -> bool:
    """K = -K (mod N), i.e. every k_i in {0, N_i/2} (§2, Fig. 1)."""
    return all(k in (0, N // 2) for k, N in zip(K, n))


def self_conjugate_points(n):
    """All K with K = -K mod N; there are 2^d of them."""
    out = []
    for K in np.ndindex(*n):
        if is_self_conjugate(K, n):
            out.append(K)
    return out


def independent_set_appendix(n):
    """The set L^N of the appendix: L_0 (all k_i in {0, M_i}) together with,
    for every split of the axes into a nonempty ordered set J = (j_1 < ... < j_m)
    and its complement, the points with k_{j_1} in 1..M-1, k_{j_i} (i > 1) in
    1..N-1 except M, and k_l in {0, M} on the complement."""
    d = len(n)
    M = [N // 2 for N in n]
    pts = set()
    for K in np.ndindex(*n):
        if all(K[i] in (0, M[i]) for i in range(d)):
            pts.add(K)
    from itertools import combinations, product
    for m in range(1, d + 1):
        for J in combinations(range(d), m):
            ranges = []
            for i in range(d):
                if i == J[0]:
                    ranges.append(range(1, M[i]))
                elif i in J:
                    ranges.append([k for k in range(1, n[i]) if k != M[i]])
                else:
                    ranges.append(sorted({0, M[i]}))
            for K in product(*ranges):
                pts.add(tuple(K))
    return pts


# ---------------------------------------------------------------------------
# Algorithm 2: Hermitian noise on the half spectrum
# ---------------------------------------------------------------------------

def alg2_normals(n: Sequence[int], seed: int):
    """(z_re, z_im) on H from the Philox mapping of Algorithm 2 (see module doc)."""
    hs = half_shape(n)
    d = len(n)
    M = n[-1] // 2
    if d == 1:
        kd = np.arange(M + 1, dtype=np.uint64)
        q = kd >> np.uint64(1)
        sel = (kd & np.uint64(1)).astype(bool)
    else:
        nmid = n[1] if d == 3 else 1
        half = np.uint64(n[0] // 2)
        k1 = np.arange(n[0], dtype=np.uint64).reshape((-1,) + (1,) * (d - 1))
        kmid = np.arange(nmid, dtype=np.uint64).reshape((1, -1, 1)) if d == 3 else np.uint64(0)
        kd = np.arange(M + 1, dtype=np.uint64).reshape((1,) * (d - 1) + (-1,))
        q = ((k1 % half) * np.uint64(nmid) + kmid) * np.uint64(M + 1) + kd
        q = np.broadcast_to(q, hs)
        sel = np.broadcast_to(k1 >= half, hs)
    w = philox_words(q, TAG_ALG2, seed)
    wa = np.where(sel, w[2], w[0])
    wb = np.where(sel, w[3], w[1])
    zr, zi = box_muller(wa, wb)
    return zr.reshape(hs), zi.reshape(hs)


def hermitian_arrangement(zr: np.ndarray, zi: np.ndarray, n: Sequence[int]) -> np.ndarray:
    """xi_K on H from normals (Lemma 1, Eq. conj, Algorithm 2, Remark on oversampling).

    * self-conjugate K:                 xi = z_re          (variance 1, real)
    * 0 < k_d < N_d/2:                  xi = (z_re + i z_im)/sqrt 2
    * k_d in {0, N_d/2}, K != -K:       the member of {K, -K} with the larger
                                        row-major index h takes (z_re + i z_im)/sqrt 2
                                        at its own index; the other takes the conjugate.
    Linear in (zr, zi); E|xi|^2 = 1 and E xi^2 = 0 off the self-conjugate points.
    """
    hs = half_shape(n)
    d = len(n)
    M = n[-1] // 2
    xi = (zr + 1j * zi) / math.sqrt(2.0)
    out = xi.copy()
    flat = np.arange(int(np.prod(hs))).reshape(hs)
    for kd in sorted({0, M}):
        # index arrays over the first d-1 axes on this plane
        for Kf in np.ndindex(*hs[:-1]) if d > 1 else [()]:
            K = tuple(Kf) + (kd,)
            Kp = negate_index(Kf, n[:-1]) + (kd,)
            if K == Kp:
                out[K] = zr[K]
            elif flat[K] < flat[Kp]:
                out[K] = np.conj(xi[Kp])
    return out


def hermitian_arrangement_vectorised(zr, zi, n):
    """Same result as hermitian_arrangement, written with array indexing (used
    for larger grids; pinned equal to the loop form by a test)."""
    hs = half_shape(n)
    d = len(n)
    M = n[-1] // 2
    xi = (zr + 1j * zi) / math.sqrt(2.0)
    out = xi.copy()
    if d == 1:
        for kd in sorted({0, M}):
            out[kd] = zr[kd]
        return out
    idx = np.indices(hs[:-1])
    neg = tuple((-idx[i]) % n[i] for i in range(d - 1))
    lead = int(np.prod(hs[:-1]))
    flat_rows = np.arange(lead).reshape(hs[:-1])
    neg_rows = flat_rows[neg]
    for kd in sorted({0, M}):
        plane = xi[..., kd]
        res = plane.copy()
        take_conj = flat_rows < neg_rows
        res[take_conj] = np.conj(plane[neg][take_conj])
        selfc = flat_rows == neg_rows
        res[selfc] = zr[..., kd][selfc]
        out[..., kd] = res
    return out


def alg2_noise(n: Sequence[int], seed: int) -> np.ndarray:
    """xi on H for one field (Algorithm 2 noise with the Philox mapping)."""
    zr, zi = alg2_normals(n, seed)
    return hermitian_arrangement_vectorised(zr, zi, n)


def extend_hermitian(AH: np.ndarray, n: Sequence[int]) -> np.ndarray:
    """Full-grid array from H using A_{-K} = conj A_K (Eq. conj)."""
    d = len(n)
    M = n[-1] // 2
    full = np.zeros(tuple(n), dtype=np.complex128)
    full[..., : M + 1] = AH
    for kd in range(M + 1, n[-1]):
        src = AH[..., n[-1] - kd]
        if d > 1:
            idx = np.indices(tuple(n[:-1]))
            neg = tuple((-idx[i]) % n[i] for i in range(d - 1))
            src = src[neg]
        full[..., kd] = np.conj(src)
    return full


# ---------------------------------------------------------------------------
# DFTs: naive O(n^2) and a recursive radix-2 FFT (both along one axis)
# ---------------------------------------------------------------------------

def dft_naive(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    """y_k = sum_j x_j exp(sign 2 pi i j k / n), unnormalised, by a dense matrix."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    nn = x.shape[-1]
    jk = np.outer(np.arange(nn), np.arange(nn)) % nn
    F = np.exp(sign * 2j * math.pi * jk / nn)
    return np.moveaxis(x @ F, -1, axis)


def fft_recursive(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    """Radix-2 decimation in time (Cooley-Tukey), recursing on the even and
    odd samples; lengths that are odd or <= 8 use the naive DFT."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    y = _fft_last(x, sign)
    return np.moveaxis(y, -1, axis)


def _fft_last(x: np.ndarray, sign: int) -> np.ndarray:
    nn = x.shape[-1]
    if nn <= 8 or nn % 2:
        return dft_naive(x, -1, sign)
    # stack even and odd samples on a new axis, transform both in one call
    eo = np.stack([x[..., 0::2], x[..., 1::2]], axis=-2)
    F = _fft_last(eo, sign)
    E, O = F[..., 0, :], F[..., 1, :]
    tw = np.exp(sign * 2j * math.pi * np.arange(nn // 2) / nn)
    return np.concatenate([E + tw * O, E - tw * O], axis=-1)


def dftn(x: np.ndarray, sign: int, naive: bool = False) -> np.ndarray:
    """d-dimensional unnormalised DFT with exp(sign 2 pi i K.j/N), axis by axis."""
    y = np.asarray(x, dtype=np.complex128)
    for ax in range(y.ndim):
        y = dft_naive(y, ax, sign) if naive else fft_recursive(y, ax, sign)
    return y


# ---------------------------------------------------------------------------
# Fields
# ---------------------------------------------------------------------------

def alg2_field_from_xi(xi: np.ndarray, n, L, spec: Spectrum, return_complex: bool = False):
    """f = IDFT(s_K xi_K) over the full grid (Eq. drf, Algorithm 2 final step)."""
    s = sqrt_scale(n, L, spec, half=True)
    full = extend_hermitian(s * xi, n)
    f = dftn(full, +1)
    return f if return_complex else f.real


def alg2_field(n, L, spec: Spectrum, seed: int, return_complex: bool = False):
    """One field by Algorithm 2 (seed is the per-field key)."""
    return alg2_field_from_xi(alg2_noise(n, seed), n, L, spec, return_complex)


def alg1_normals(n: Sequence[int], seed: int) -> np.ndarray:
    """Real N(0,1) noise on the full grid from the Philox mapping of Algorithm 1."""
    ntot = int(np.prod(n))
    j = np.arange(ntot, dtype=np.uint64)
    w = philox_words(j >> np.uint64(2), TAG_ALG1, seed)
    t = ((j & np.uint64(3)) >> np.uint64(1)).astype(bool)
    wa = np.where(t, w[2], w[0])
    wb = np.where(t, w[3], w[1])
    zr, zi = box_muller(wa, wb)
    odd = (j & np.uint64(1)).astype(bool)
    return np.where(odd, zi, zr).reshape(tuple(n))


def alg1_field_from_z(z: np.ndarray, n, L, spec: Spectrum, return_complex: bool = False):
    """f = IDFT( s_K DFT(z)_K / sqrt(N_tot) ) (Eq. 1, Algorithm 1)."""
    ntot = int(np.prod(n))
    s = sqrt_scale(n, L, spec)
    Z = dftn(z, -1)
    f = dftn(s * Z / math.sqrt(ntot), +1)
    return f if return_complex else f.real


def alg1_field(n, L, spec: Spectrum, seed: int, return_complex: bool = False):
    return alg1_field_from_z(alg1_normals(n, seed), n, L, spec, return_complex)


def sample(n, L, spec: Spectrum, seed: int, batch: int = 1, alg: int = ALG_ONE_FFT) -> np.ndarray:
    """batch fields; field b uses key seed + b."""
    fn = alg2_field if alg == ALG_ONE_FFT else alg1_field
    return np.stack([fn(n, L, spec, (seed + b) & 0xFFFFFFFFFFFFFFFF) for b in range(batch)])


# --- sampled outputs at large sizes -----------------------------------------

def alg2_halfspectrum(n, L, spec: Spectrum, seed: int) -> np.ndarray:
    """A_K = s_K xi_K on H."""
    return sqrt_scale(n, L, spec, half=True) * alg2_noise(n, seed)


def field_lines(AH: np.ndarray, n, lead_index_list) -> np.ndarray:
    """Selected lines f[j_1, ..., j_{d-1}, :] of the field with half spectrum AH,
    by the definition f_j = sum_K A_K exp(+2 pi i K.j/N): the sum over
    k_1..k_{d-1} is a dense contraction for each chosen (j_1..j_{d-1}), the sum
    over k_d a 1-D inverse DFT of the Hermitian-extended line."""
    d = len(n)
    M = n[-1] // 2
    out = []
    for J in lead_index_list:
        line = AH
        for i in range(d - 1):
            e = np.exp(2j * math.pi * np.arange(n[i]) * J[i] / n[i])
            line = np.tensordot(e, line, axes=([0], [0]))
        full = np.zeros(n[-1], dtype=np.complex128)
        full[: M + 1] = line
        full[M + 1:] = np.conj(line[1:M][::-1]) if M > 1 else full[M + 1:]
        out.append(fft_recursive(full, 0, +1).real)
    return np.stack(out)


# ---------------------------------------------------------------------------
# Exact covariance
# ---------------------------------------------------------------------------

def exact_covariance(n, L, spec: Spectrum) -> np.ndarray:
    """c(r) = (1/|D|) sum_K S(p_K) cos(2 pi K.r/N) on the grid of lags r."""
    S = scaled_density(n, L, spec)
    return dftn(S, +1).real


def covariance_bruteforce(n, L, spec: Spectrum) -> np.ndarray:
    """Dense N_tot x N_tot matrix Sigma_{jl} = c(j - l), summed term by term."""
    S = scaled_density(n, L, spec).ravel()
    Ks = np.array(list(np.ndindex(*n)), dtype=np.float64)
    js = Ks.copy()
    nn = np.array(n, dtype=np.float64)
    ph = 2 * math.pi * (Ks / nn) @ js.T  # K . j / N
    # Sigma_{jl} = sum_K S_K cos(2 pi K.(j - l)/N)
    C = np.cos(ph).T * S @ np.cos(ph) + np.sin(ph).T * S @ np.sin(ph)
    return C


# ---------------------------------------------------------------------------
# Loss on the radially binned power spectrum and its gradient
# ---------------------------------------------------------------------------

def digamma(x: float) -> float:
    """psi(x) by the recurrence psi(x) = psi(x+1) - 1/x up to x >= 6 and the
    asymptotic series psi(x) ~ ln x - 1/(2x) - sum B_2k / (2k x^2k)
    (Abramowitz & Stegun 6.3.5 and 6.3.18)."""
    acc = 0.0
    while x < 10.0:
        acc -= 1.0 / x
        x += 1.0
    x2 = 1.0 / (x * x)
    series = x2 * (1.0 / 12 - x2 * (1.0 / 120 - x2 * (1.0 / 252 - x2 * (1.0 / 240 - x2 * (1.0 / 132)))))
    return acc + math.log(x) - 0.5 / x - series


def half_weights(n) -> np.ndarray:
    """w_K on H: 1 on the planes k_d in {0, N_d/2}, 2 elsewhere (each such K stands for K and -K)."""
    hs = half_shape(n)
    w = np.full(hs, 2.0)
    w[..., 0] = 1.0
    w[..., n[-1] // 2] = 1.0
    return w


def dlogS(n, L, spec: Spectrum):
    """d log S / d(sigma, ell, nu) on H (Matern and Gaussian)."""
    d = len(n)
    p = frequency_grid(n, L, half=True)
    p2 = sum(pi ** 2 for pi in p)
    ds = np.full(p2.shape, 2.0 / spec.sigma)
    if spec.family == MATERN:
        w2 = (2 * math.pi) ** 2 * p2
        a = spec.nu + d / 2.0
        den = 1.0 + spec.ell ** 2 * w2
        dl = d / spec.ell - a * 2.0 * spec.ell * w2 / den
        dn = digamma(a) - digamma(spec.nu) - np.log(den)
    elif spec.family == GAUSSIAN:
        dl = d / spec.ell - 4.0 * math.pi ** 2 * spec.ell * p2
        dn = np.zeros_like(p2)
    else:
        raise ValueError("gradient only for Matern and Gaussian")
    if spec.normalize_discrete:
        raise ValueError("gradient not defined with normalize_discrete")
    return ds, dl, dn


@dataclass
class BinnedLossSpec:
    nbins: int = 64
    target: Spectrum = field(default_factory=lambda: Spectrum(MATERN, 1.0, 0.08, 2.0))


def radial_bins(n, L, nbins: int):
    """Bin index of every H entry (-1 for |p| >= p_max, p_max = min_i N_i/(2 L_i))."""
    p = frequency_grid(n, L, half=True)
    pm = np.sqrt(sum(pi ** 2 for pi in p))
    pmax = min(N / (2.0 * Li) for N, Li in zip(n, L))
    b = np.floor(pm / pmax * nbins).astype(np.int64)
    b[pm >= pmax] = -1
    return b


def binned_power(P_H: np.ndarray, bins: np.ndarray, w: np.ndarray, nbins: int):
    """Weighted mean of P over each bin, and the bin weights W_b."""
    m = bins >= 0
    Wb = np.bincount(bins[m], weights=w[m], minlength=nbins)
    Sb = np.bincount(bins[m], weights=(w * P_H)[m], minlength=nbins)
    return Sb / np.where(Wb > 0, Wb, 1.0), Wb


def power_loss_from_fields(fields: np.ndarray, n, L, loss: BinnedLossSpec) -> float:
    """L = (1/B) sum_fields sum_b (P_b - T_b)^2 with P_K = |DFT(f)_K|^2 / N_tot^2 on H."""
    B = fields.shape[0]
    ntot = int(np.prod(n))
    bins = radial_bins(n, L, loss.nbins)
    w = half_weights(n)
    T, _ = binned_power(scaled_density(n, L, loss.target, half=True), bins, w, loss.nbins)
    M = n[-1] // 2
    tot = 0.0
    for b in range(B):
        F = dftn(fields[b], -1)[..., : M + 1]
        P, _ = binned_power(np.abs(F) ** 2 / ntot ** 2, bins, w, loss.nbins)
        tot += float(((P - T) ** 2).sum())
    return tot / B


def power_loss_and_grad(n, L, spec: Spectrum, seed: int, batch: int, loss: BinnedLossSpec):
    """Loss of the Algorithm 2 fields (seeds seed..seed+batch-1) and its analytic
    gradient d L / d(sigma, ell, nu):
        dL/dtheta = (2/B) sum_fields sum_b (P_b - T_b) (sum_{K in b} w_K |xi_K|^2 d_theta(s_K^2)) / W_b,
    with d_theta(s_K^2) = s_K^2 d_theta log S (P_K = |A_K|^2 = s_K^2 |xi_K|^2 exactly)."""
    bins = radial_bins(n, L, loss.nbins)
    w = half_weights(n)
    s2 = scaled_density(n, L, spec, half=True)
    T, Wb = binned_power(scaled_density(n, L, loss.target, half=True), bins, w, loss.nbins)
    dls = dlogS(n, L, spec)
    m = bins >= 0
    Lval = 0.0
    g = np.zeros(3)
    for b in range(batch):
        xi2 = np.abs(alg2_noise(n, (seed + b) & 0xFFFFFFFFFFFFFFFF)) ** 2
        P, _ = binned_power(s2 * xi2, bins, w, loss.nbins)
        diff = P - T
        Lval += float((diff ** 2).sum())
        for t in range(3):
            num = np.bincount(bins[m], weights=(w * xi2 * s2 * dls[t])[m], minlength=loss.nbins)
            g[t] += 2.0 * float((diff * num / np.where(Wb > 0, Wb, 1.0)).sum())
    return Lval / batch, g / batch


def adjoint_grad(n, L, spec: Spectrum, seed: int, grad_fields: np.ndarray) -> np.ndarray:
    """Per field: dLoss/dtheta = sum_j G_j d f_j / d theta for an upstream
    gradient G (real field), Algorithm 2.  Since f = IDFT(s xi),
    d f / d theta = IDFT(d_theta s xi), and with G^ = DFT(G) (exp(-)):
        sum_j G_j df_j/dtheta = sum_{K in H} w_K d_theta s_K Re(xi_K conj(G^_K)).
    Returns an array (batch, 3)."""
    s = sqrt_scale(n, L, spec, half=True)
    dls = dlogS(n, L, spec)
    w = half_weights(n)
    M = n[-1] // 2
    out = np.zeros((grad_fields.shape[0], 3))
    for b in range(grad_fields.shape[0]):
        xi = alg2_noise(n, (seed + b) & 0xFFFFFFFFFFFFFFFF)
        G = dftn(grad_fields[b], -1)[..., : M + 1]
        re = (xi * np.conj(G)).real
        for t in range(3):
            out[b, t] = float((w * 0.5 * s * dls[t] * re).sum())
    return out


def rfft_halfspectrum(x: np.ndarray) -> np.ndarray:
    """DFT (exp(-)) of a real d-dimensional array, restricted to H."""
    M = x.shape[-1] // 2
    return dftn(x, -1)[..., : M + 1]


# ---------------------------------------------------------------------------
# Boundary-condition variants: cosine (Neumann) and sine (Dirichlet) transforms
# ---------------------------------------------------------------------------
#
# §1 and §3 remark that the FFT may be replaced by the fast cosine or sine
# transform, which gives fields with Neumann or Dirichlet boundary conditions;
# the paper gives no formulas.  The reading fixed here:
#
# * the box [0, L_1] x ... x [0, L_d] carries N_i intervals per axis (N_i a
#   power of two), i.e. the N_i + 1 points x_j = j L_i / N_i, j = 0..N_i;
# * the spectral density is sampled on the frequencies of the mirrored box of
#   edges 2 L_i (the even or odd extension of the field is periodic there):
#   p_K = (k_i / (2 L_i))_i, k_i = 0..N_i, and S(p_K) / |2D|, |2D| = prod 2 L_i;
# * Neumann: f_J = sum_{K in prod{0..N_i}} sqrt(w_K S(p_K)/|2D|) a_K prod_i cos(pi k_i j_i / N_i),
#   w_K = prod_i w(k_i), w = 1 at k in {0, N}, 2 inside (the number of points
#   of the mirrored grid that k stands for);
# * Dirichlet: the same with sin(pi k_i j_i / N_i) and K over the interior
#   prod{1..N_i-1} (w_K = 2^d); f vanishes on the boundary faces;
# * a_K are independent N(0,1) reals; with the flat row-major index j of K in
#   the (N_1+1) x ... x (N_d+1) grid: call j >> 2, counter (q_lo, q_hi, 2, 0),
#   words 2t, 2t+1 with t = (j & 3) >> 1, even j the cosine normal of
#   Box-Muller, odd j the sine normal (Algorithm 1's mapping with tag 2).
# The covariance of either field is then the method-of-images sum of the
# periodic covariance c of the mirrored grid (2 N_i points, period 2 L_i):
#   Cov(f_J, f_J') = 2^-d sum_{sigma in {+1,-1}^d} sgn(sigma) c(J + sigma J'),
# sgn = 1 (Neumann) or prod_i (-sigma_i) (Dirichlet); the tests pin the oracle
# to that identity.

BC_NEUMANN = 1
BC_DIRICHLET = 2
TAG_BC = 2


def bc_shape(n: Sequence[int]):
    """Points per axis of a boundary-condition field: N_i + 1."""
    return tuple(int(x) + 1 for x in n)


def bc_normals(n: Sequence[int], seed: int) -> np.ndarray:
    """Real N(0,1) a_K on prod{0..N_i}: call j >> 2 (tag 2), pair (j & 3) >> 1, even j cos, odd j sin."""
    shp = bc_shape(n)
    ntot = int(np.prod(shp))
    j = np.arange(ntot, dtype=np.uint64)
    w = philox_words(j >> np.uint64(2), TAG_BC, seed)
    t = ((j & np.uint64(3)) >> np.uint64(1)).astype(bool)
    wa = np.where(t, w[2], w[0])
    wb = np.where(t, w[3], w[1])
    zr, zi = box_muller(wa, wb)
    odd = (j & np.uint64(1)).astype(bool)
    return np.where(odd, zi, zr).reshape(shp)


def bc_axis_matrix(N: int, bc: int) -> np.ndarray:
    """E[j, k] = cos(pi k j / N) (Neumann) or sin(pi k j / N) (Dirichlet), j, k = 0..N.

    The angle is reduced exactly first: with m = k j mod 2N, pi k j / N = pi m / N
    (mod 2 pi); the values at the quarter points m in {0, N/2, N, 3N/2} are
    set to their exact 0 / +-1, so that the sine rows j in {0, N} vanish exactly."""
    k = np.arange(N + 1, dtype=np.int64)
    m = np.outer(k, k) % (2 * N)  # symmetric in (j, k)
    ang = math.pi * m.astype(np.float64) / N
    if bc == BC_NEUMANN:
        E = np.cos(ang)
        E[m == 0] = 1.0
        E[m == N] = -1.0
        if N % 2 == 0:
            E[(m == N // 2) | (m == 3 * N // 2)] = 0.0
    elif bc == BC_DIRICHLET:
        E = np.sin(ang)
        E[(m == 0) | (m == N)] = 0.0
        if N % 2 == 0:
            E[m == N // 2] = 1.0
            E[m == 3 * N // 2] = -1.0
    else:
        raise ValueError("unknown boundary condition")
    return E


def bc_weights(n: Sequence[int], bc: int) -> np.ndarray:
    """w_K on prod{0..N_i}: Neumann prod w(k_i) with w = 1 at {0, N}, 2 inside;
    Dirichlet 2^d inside and 0 on the boundary."""
    w = np.ones(bc_shape(n))
    for i, N in enumerate(n):
        wi = np.full(N + 1, 2.0)
        wi[0] = wi[N] = 1.0 if bc == BC_NEUMANN else 0.0
        shape = [1] * len(n)
        shape[i] = N + 1
        w = w * wi.reshape(shape)
    return w


def bc_scaled_density(n: Sequence[int], L: Sequence[float], spec: Spectrum) -> np.ndarray:
    """S(p_K) / |2D| with p_K = (k_i / (2 L_i))_i, k_i = 0..N_i (the mirrored box)."""
    if spec.normalize_discrete:
        raise ValueError("normalize_discrete is not defined for boundary-condition fields")
    axes = [np.arange(N + 1, dtype=np.float64) / (2.0 * Li) for N, Li in zip(n, L)]
    p = np.meshgrid(*axes, indexing="ij")
    vol2 = float(np.prod([2.0 * Li for Li in L]))
    return spectral_density(p, spec) / vol2


def bc_coefficients(n, L, spec: Spectrum, bc: int) -> np.ndarray:
    """sqrt(w_K S(p_K) / |2D|), the factor in front of a_K."""
    return np.sqrt(bc_weights(n, bc) * bc_scaled_density(n, L, spec))


def bc_field_from_a(a: np.ndarray, n, L, spec: Spectrum, bc: int) -> np.ndarray:
    """f_J = sum_K coef_K a_K prod_i E_i[j_i, k_i], one axis at a time (a dense
    (N_i+1) x (N_i+1) matrix product per axis)."""
    x = bc_coefficients(n, L, spec, bc) * a
    for i, N in enumerate(n):
        E = bc_axis_matrix(N, bc)
        x = np.moveaxis(np.tensordot(E, x, axes=([1], [i])), 0, i)
    return x


def bc_field(n, L, spec: Spectrum, bc: int, seed: int) -> np.ndarray:
    """One Neumann or Dirichlet field (seed is the per-field key)."""
    return bc_field_from_a(bc_normals(n, seed), n, L, spec, bc)


def bc_sample(n, L, spec: Spectrum, bc: int, seed: int, batch: int = 1) -> np.ndarray:
    """batch fields; field b uses key seed + b."""
    return np.stack([bc_field(n, L, spec, bc, (seed + b) & 0xFFFFFFFFFFFFFFFF) for b in range(batch)])


def bc_field_lines(n, L, spec: Spectrum, bc: int, seed: int, lead_index_list) -> np.ndarray:
    """Selected lines f[j_1, ..., j_{d-1}, :] of one field, by the same sums:
    for each chosen (j_1..j_{d-1}) the sums over k_1..k_{d-1} contract against
    the rows E_i[j_i, :], then the last axis is a dense matrix product."""
    x = bc_coefficients(n, L, spec, bc) * bc_normals(n, seed)
    Ed = bc_axis_matrix(n[-1], bc)
    out = []
    for J in lead_index_list:
        line = x
        for i in range(len(n) - 1):
            line = np.tensordot(bc_axis_matrix(n[i], bc)[J[i]], line, axes=([0], [0]))
        out.append(Ed @ line)
    return np.stack(out)


def bc_exact_covariance(n, L, spec: Spectrum, bc: int, J, Jp) -> float:
    """Cov(f_J, f_J') by the method of images on the mirrored periodic grid:
    2^-d sum_sigma sgn(sigma) c(J + sigma J') with c = exact_covariance(2n, 2L)."""
    d = len(n)
    n2 = [2 * N for N in n]
    c = exact_covariance(n2, [2.0 * Li for Li in L], spec)
    acc = 0.0
    for sig in np.ndindex(*([2] * d)):
        s = [1 if t == 0 else -1 for t in sig]
        lag = tuple((J[i] + s[i] * Jp[i]) % n2[i] for i in range(d))
        sgn = 1.0 if bc == BC_NEUMANN else float(np.prod([-si for si in s]))
        acc += sgn * c[lag]
    return acc / 2 ** d
