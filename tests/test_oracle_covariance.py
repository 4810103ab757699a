"""Pins for what the oracle's fields are: brute-force covariance of the linear
map from noise to field (both algorithms), closed-form covariances (Gaussian,
Matern 1/2, 3/2, 5/2, and the paper's own 1-D example of §4), and a Monte
Carlo check with exact confidence bands."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import grf_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")

SPECS = [O.Spectrum(O.MATERN, 1.3, 0.2, 1.5), O.Spectrum(O.GAUSSIAN, 0.7, 0.15, 0.0),
         O.Spectrum(O.MATERN, 1.0, 0.3, 0.5)]


def _alg2_linear_map(n, L, spec):
    hs = O.half_shape(n)
    cols = []
    for part in (0, 1):
        for K in np.ndindex(*hs):
            zr, zi = np.zeros(hs), np.zeros(hs)
            (zr if part == 0 else zi)[K] = 1.0
            xi = O.hermitian_arrangement_vectorised(zr, zi, n)
            cols.append(O.alg2_field_from_xi(xi, n, L, spec).ravel())
    return np.array(cols).T


def _alg1_linear_map(n, L, spec):
    ntot = int(np.prod(n))
    cols = []
    for j in range(ntot):
        z = np.zeros(ntot)
        z[j] = 1.0
        cols.append(O.alg1_field_from_z(z.reshape(n), n, L, spec).ravel())
    return np.array(cols).T


@pytest.mark.parametrize("n,L", [((8,), (1.0,)), ((8, 8), (1.0, 1.0)), ((4, 6), (0.7, 1.9)),
                                 ((4, 4, 4), (1.0, 1.0, 1.0)), ((2, 4, 6), (1.0, 2.0, 0.5)), ((2,), (1.0,)),
                                 ((10,), (1.3,)), ((14,), (2.0,)), ((6, 10), (1.0, 0.8))])
@pytest.mark.parametrize("si", range(len(SPECS)))
def test_linear_map_covariance_is_circulant(n, L, si):
    spec = SPECS[si]
    Sigma = O.covariance_bruteforce(n, L, spec)
    for Mmap in (_alg2_linear_map(n, L, spec), _alg1_linear_map(n, L, spec)):
        np.testing.assert_allclose(Mmap @ Mmap.T, Sigma, atol=1e-12 * np.abs(Sigma).max())
    # the first row of Sigma is the exact covariance c(r)
    np.testing.assert_allclose(Sigma[0], O.exact_covariance(n, L, spec).ravel(), atol=1e-12)


def _lags(N, L):
    r = np.arange(N) * (L / N)
    return np.minimum(r, L - r)


@pytest.mark.parametrize("n", [(64,), (64, 32), (64, 64, 64)])
def test_gaussian_closed_form(n):
    ell = 0.05
    L = tuple(1.0 if N == 64 else 0.5 for N in n)
    spec = O.Spectrum(O.GAUSSIAN, 1.0, ell, 0.0)
    c = O.exact_covariance(n, L, spec)
    # the periodised closed form is a product of 1-D image sums
    per = [sum(np.exp(-(_lags(N, Li) + m * Li) ** 2 / (2 * ell ** 2)) for m in range(-3, 4))
           for N, Li in zip(n, L)]
    want = per[0]
    for p1 in per[1:]:
        want = np.multiply.outer(want, p1)
    np.testing.assert_allclose(c, want, atol=1e-12)


MATERN_CLOSED = {
    0.5: lambda x: np.exp(-x),
    1.5: lambda x: (1 + x) * np.exp(-x),
    2.5: lambda x: (1 + x + x ** 2 / 3) * np.exp(-x),
}


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_closed_form_within_tail_bound(nu):
    N, Lx, ell = 4096, 1.0, 0.02
    spec = O.Spectrum(O.MATERN, 1.0, ell, nu)
    c = O.exact_covariance((N,), (Lx,), spec)
    r = _lags(N, Lx)
    Cper = sum(MATERN_CLOSED[nu](np.abs(r + m * Lx) / ell) for m in range(-3, 4))
    # |c - C_per| <= (1/L) sum_{|k| > N/2} S(k/L) (the periodised continuum covariance
    # keeps every frequency k/L; the grid keeps -N/2 < k <= N/2, so k = -N/2 is missing too)
    S = lambda k: O.spectral_density([np.asarray(k, dtype=np.float64) / Lx], spec) / Lx
    k0, K = N // 2, 2 ** 22
    # sum_{k > k0} S(k) <= sum_{k0 < k < K} S(k) + S(K) + int_K^inf C k^-2a dk, where
    # C k^-2a >= S(k) with a = nu + 1/2 and C = c/L (2 pi ell / L)^-2a
    a = nu + 0.5
    Cc = O.matern_constant(ell, nu, 1) / Lx * (2 * math.pi * ell / Lx) ** (-2 * a)
    one_side = S(np.arange(k0 + 1, K)).sum() + S(K) + Cc * K ** (1 - 2 * a) / (2 * a - 1)
    tail = float(S(k0) + 2 * one_side)
    err = np.abs(c - Cper).max()
    assert err <= tail + 1e-12, (err, tail)
    # the bound is not vacuous: c(0) is close to 1
    assert abs(c[0] - 1.0) <= tail + 1e-12


def _paper_example():
    vals = {}
    with open(os.path.join(GOLD, "paper_1d_example.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, *v = ln.split()
                vals[k] = [float(Fraction(x)) for x in v]
    return vals


def test_paper_1d_example_spectrum_is_matern_7_2():
    """The paper's gamma (angular frequency) equals, in cycles, the Matern density with
    nu = 7/2, ell = 1/10: S(p) = 2 pi gamma(2 pi p)."""
    g = _paper_example()
    spec = O.Spectrum(O.MATERN, 1.0, 0.1, 3.5)
    p = np.linspace(-20, 20, 101)
    gamma = lambda w: g["gamma_const"][0] / math.pi / (g["gamma_shift"][0] + w ** 2) ** g["gamma_power"][0]
    np.testing.assert_allclose(O.spectral_density([p], spec), 2 * math.pi * gamma(2 * math.pi * p), rtol=1e-13)


def test_paper_1d_example_convergence():
    g = _paper_example()
    a = g["C_coeffs"]
    rate = g["C_rate"][0]
    C = lambda r: (a[0] + a[1] * r + a[2] * r ** 2 + a[3] * r ** 3) * np.exp(-rate * r)
    Lx = g["domain_hi"][0] - g["domain_lo"][0]
    spec = O.Spectrum(O.MATERN, 1.0, 0.1, 3.5)
    errs = {}
    for nexp in range(int(g["n_min"][0]), int(g["n_max"][0]) + 1):
        N = 2 ** nexp
        c = O.exact_covariance((N,), (Lx,), spec)
        i = np.arange(-N // 2, N // 2 + 1)
        x = i * math.pi / 2 ** (nexp - 1)
        cn = c[i % N]
        errs[N] = np.abs(cn - C(np.abs(x))).max()
    # the error falls on every refinement until it reaches the periodisation floor
    # (the torus keeps the images C(x + 2 pi m); the paper compares with C itself)
    floor = 2.5 * C(math.pi)
    for N in [4, 8, 16, 32, 64, 128, 256]:
        assert errs[2 * N] < errs[N]
    # and, once the grid resolves the spectrum, at least like N^-4 (Figure 8 ends at n = 6, N = 64)
    for N in [16, 32]:
        assert math.log2(errs[N] / errs[2 * N]) >= -g["order"][0], (N, errs[N], errs[2 * N])
    assert errs[4096] <= floor


def test_normalize_discrete_gives_exact_variance():
    spec = O.Spectrum(O.MATERN, 1.7, 0.3, 0.5, normalize_discrete=1)
    c = O.exact_covariance((16, 8), (1.0, 1.0), spec)
    assert abs(c[0, 0] - 1.7 ** 2) < 1e-12


@pytest.mark.parametrize("alg", [1, 2])
def test_monte_carlo_covariance_bands(alg):
    n, L = (16, 16), (1.0, 1.0)
    spec = O.Spectrum(O.MATERN, 1.0, 0.1, 1.5)
    Mf = 1200
    fs = O.sample(n, L, spec, seed=1000 * alg, batch=Mf, alg=alg)
    c = O.exact_covariance(n, L, spec)
    ntot = 256
    for r in [(0, 0), (1, 0), (0, 1), (2, 3), (8, 8)]:
        est = np.mean(fs * np.roll(fs, shift=(-r[0], -r[1]), axis=(1, 2)))
        cr = c[r]
        cp = np.roll(c, shift=(-r[0], -r[1]), axis=(0, 1))
        cm = np.roll(c, shift=(r[0], r[1]), axis=(0, 1))
        var = float((c ** 2 + cp * cm).sum()) / (Mf * ntot)
        assert abs(est - cr) <= 5 * math.sqrt(var), (r, est, cr, math.sqrt(var))
