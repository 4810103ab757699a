"""Pins of the oracle's polynomial family of §4,
gamma(p) = sigma^2 (m^(k l) + (p_1^(2k) + p_2^(2k))^l)^(-n):

* k = l = 1, n = 2 in 2-D is the Matern density with nu = 1: with
  ell = 1 / (2 pi sqrt m) and sigma_M^2 = pi / m the two coincide (Matern's
  constant (2 sqrt(pi) ell)^2 Gamma(2) / Gamma(1) = 4 pi ell^2 = 1 / (pi m));
* its integral over R^2 for k = l = 1 is the closed form pi / ((n - 1) m^(n-1)),
  for k = 1, l = 2, n = 1 it is pi^2 / (2 m), and for k = 2, l = 1, n = 1 it is
  pi K(1/2) / m (complete elliptic integral), checked by polar quadrature;
* the exponents: m enters as m^(k l), the sum of p_i^(2k) is raised to l and the
  whole to -n (the value at p = 0 is m^(-k l n); on the axis p = (t, 0) it is
  (m^(k l) + t^(2 k l))^(-n));
* symmetry: even in each p_i and under the swap p_1 <-> p_2; rotation invariant
  only for k = 1 (Fig. 3(d), k = 3, is anisotropic)."""
import math

import numpy as np
import pytest

from oracle import grf_oracle as O


def _S(spec, p1, p2):
    return O.spectral_density([np.asarray(p1, float), np.asarray(p2, float)], spec)


@pytest.mark.parametrize("m", [0.75, 2.0, 10.0])
def test_k1_l1_n2_is_matern_nu1(m):
    poly = O.Spectrum(O.PAPER_POLY, sigma=1.0, m=m, k=1, l=1, n=2)
    mat = O.Spectrum(O.MATERN, sigma=math.sqrt(math.pi / m), ell=1.0 / (2 * math.pi * math.sqrt(m)), nu=1.0)
    rng = np.random.default_rng(1)
    p1, p2 = rng.normal(scale=3.0, size=(2, 200))
    np.testing.assert_allclose(_S(poly, p1, p2), _S(mat, p1, p2), rtol=1e-12)


@pytest.mark.parametrize("m,n", [(2.0, 2), (10.0, 3), (0.75, 2)])
def test_integral_closed_form(m, n):
    """int_{R^2} (m + |p|^2)^(-n) dp = pi / ((n - 1) m^(n - 1)), by the radial
    integral 2 pi int_0^inf r (m + r^2)^(-n) dr on a substituted grid."""
    spec = O.Spectrum(O.PAPER_POLY, sigma=1.0, m=m, k=1, l=1, n=n)
    # r = sqrt(m) tan(theta), theta in (0, pi/2): dr = sqrt(m) sec^2 dtheta
    th = (np.arange(200000) + 0.5) * (math.pi / 2) / 200000
    r = math.sqrt(m) * np.tan(th)
    integrand = 2 * math.pi * r * _S(spec, r, 0.0 * r) * math.sqrt(m) / np.cos(th) ** 2
    val = integrand.sum() * (math.pi / 2) / 200000
    assert math.isclose(val, math.pi / ((n - 1) * m ** (n - 1)), rel_tol=1e-6)


def _polar_integral(spec, nr=40000, nt=256, scale=1.0):
    """int_{R^2} S dp in polar coordinates: theta by the midpoint rule
    (periodic, spectrally accurate), r = scale tan(phi) with the midpoint rule
    in phi on (0, pi/2)."""
    ph = (np.arange(nr) + 0.5) * (math.pi / 2) / nr
    r = scale * np.tan(ph)
    w_r = r * scale / np.cos(ph) ** 2 * (math.pi / 2) / nr
    th = (np.arange(nt) + 0.5) * 2 * math.pi / nt
    tot = 0.0
    for t in th:
        tot += float((_S(spec, r * math.cos(t), r * math.sin(t)) * w_r).sum())
    return tot * 2 * math.pi / nt


@pytest.mark.parametrize("m", [0.75, 10.0])
def test_l2_integral_closed_form(m):
    """k = 1, l = 2, n = 1 (Fig. 3 (a), (b)): int (m^2 + |p|^4)^(-1) dp = pi^2 / (2 m)."""
    spec = O.Spectrum(O.PAPER_POLY, sigma=1.0, m=m, k=1, l=2, n=1)
    val = _polar_integral(spec, nt=8, scale=math.sqrt(m))
    assert math.isclose(val, math.pi ** 2 / (2 * m), rel_tol=1e-6)


@pytest.mark.parametrize("m", [1.0, 5.0])
def test_k2_integral_is_elliptic(m):
    """k = 2, l = 1, n = 1: int (m^2 + p_1^4 + p_2^4)^(-1) dp = pi K(1/2) / m,
    K the complete elliptic integral of the first kind (parameter 1/2): the
    radial integral gives pi / (4 m sqrt(1 - sin^2(2 theta) / 2)), whose angular
    integral is 4 K(1/2)."""
    special = pytest.importorskip("scipy.special")
    spec = O.Spectrum(O.PAPER_POLY, sigma=1.0, m=m, k=2, l=1, n=1)
    val = _polar_integral(spec, nt=512, scale=math.sqrt(m))
    assert math.isclose(val, math.pi * float(special.ellipk(0.5)) / m, rel_tol=1e-6)


@pytest.mark.parametrize("m,k,l,n", [(10.0, 1, 2, 1), (0.75, 1, 2, 1), (10.0, 1, 1, 3), (5.0, 3, 1, 1), (2.0, 2, 3, 2)])
def test_exponent_placement(m, k, l, n):
    spec = O.Spectrum(O.PAPER_POLY, sigma=1.7, m=m, k=k, l=l, n=n)
    assert math.isclose(float(_S(spec, 0.0, 0.0)), 1.7 ** 2 * m ** (-k * l * n), rel_tol=1e-13)
    for t in (0.3, 1.0, 2.5):
        want = 1.7 ** 2 * (m ** (k * l) + t ** (2 * k * l)) ** (-n)
        assert math.isclose(float(_S(spec, t, 0.0)), want, rel_tol=1e-13)
        # on the diagonal p = (t, t): (m^(k l) + (2 t^(2k))^l)^(-n)
        want_d = 1.7 ** 2 * (m ** (k * l) + (2 * t ** (2 * k)) ** l) ** (-n)
        assert math.isclose(float(_S(spec, t, t)), want_d, rel_tol=1e-13)


@pytest.mark.parametrize("k", [1, 3])
def test_symmetries(k):
    spec = O.Spectrum(O.PAPER_POLY, sigma=1.0, m=5.0, k=k, l=1, n=1)
    rng = np.random.default_rng(2)
    p1, p2 = rng.normal(size=(2, 100))
    base = _S(spec, p1, p2)
    for q1, q2 in [(-p1, p2), (p1, -p2), (p2, p1)]:
        np.testing.assert_allclose(_S(spec, q1, q2), base, rtol=1e-14)
    # rotation by 45 degrees: invariant for k = 1 only
    c = math.sqrt(0.5)
    rot = _S(spec, c * (p1 - p2), c * (p1 + p2))
    if k == 1:
        np.testing.assert_allclose(rot, base, rtol=1e-12)
    else:
        assert np.max(np.abs(rot - base) / base) > 1e-2
