"""Pins of the oracle's boundary-condition variants (the cosine / sine
transform remark of §1 and §3): the per-axis transforms against scipy's DCT-I
and DST-I, the covariance of the sampled law against the method-of-images sum
of the periodic covariance on the mirrored grid (brute force over the linear
map), exact zeros on Dirichlet faces, and the moments of the real noise."""

import math

import numpy as np
import pytest

from oracle import grf_oracle as o

scipy_fft = pytest.importorskip("scipy.fft")


@pytest.mark.parametrize("N", [2, 4, 8, 16, 64])
def test_cosine_matrix_is_dct1(N):
    """sum_k c_k cos(pi k j / N) = DCT-I of (c_0, c_1/2, ..., c_{N-1}/2, c_N)."""
    rng = np.random.default_rng(N)
    c = rng.standard_normal(N + 1)
    x = c.copy()
    x[1:N] *= 0.5
    ref = scipy_fft.dct(x, type=1)
    got = o.bc_axis_matrix(N, o.BC_NEUMANN) @ c
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(c).sum())


@pytest.mark.parametrize("N", [2, 4, 8, 16, 64])
def test_sine_matrix_is_dst1(N):
    """sum_k c_k sin(pi k j / N) over the interior = DST-I(c_1..c_{N-1}) / 2, and 0 at j in {0, N}."""
    rng = np.random.default_rng(100 + N)
    c = rng.standard_normal(N + 1)
    E = o.bc_axis_matrix(N, o.BC_DIRICHLET)
    got = E @ c
    ref = scipy_fft.dst(c[1:N], type=1) / 2
    np.testing.assert_allclose(got[1:N], ref, rtol=0, atol=1e-12 * np.abs(c).sum())
    assert got[0] == 0.0 and got[N] == 0.0
    # the boundary coefficients k in {0, N} do not enter
    assert np.all(E[:, 0] == 0.0) and np.all(E[:, N] == 0.0)


def _linear_map(n, L, spec, bc):
    """Dense matrix B with f = B a (columns: the field of each unit noise vector)."""
    shp = o.bc_shape(n)
    ntot = int(np.prod(shp))
    B = np.empty((ntot, ntot))
    for q in range(ntot):
        e = np.zeros(ntot)
        e[q] = 1.0
        B[:, q] = o.bc_field_from_a(e.reshape(shp), n, L, spec, bc).ravel()
    return B


CASES = [
    ((8,), (1.3,), o.Spectrum(family=o.MATERN, sigma=1.2, ell=0.2, nu=1.5)),
    ((16,), (2.0,), o.Spectrum(family=o.GAUSSIAN, sigma=0.8, ell=0.15)),
    ((4, 8), (1.0, 2.5), o.Spectrum(family=o.MATERN, sigma=1.0, ell=0.3, nu=0.5)),
    ((8, 4), (0.7, 1.1), o.Spectrum(family=o.PAPER_POLY, sigma=1.0, m=2.0, k=2, l=1, n=2)),
    ((2, 4, 4), (1.0, 0.5, 2.0), o.Spectrum(family=o.GAUSSIAN, sigma=1.0, ell=0.25)),
]


@pytest.mark.parametrize("bc", [o.BC_NEUMANN, o.BC_DIRICHLET])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_covariance_is_image_sum(case, bc):
    """Cov = B B^T of the linear map equals 2^-d sum_sigma sgn c(J + sigma J') of
    the periodic covariance on the mirrored grid (2 N_i points, period 2 L_i)."""
    n, L, spec = CASES[case]
    B = _linear_map(n, L, spec, bc)
    Sig = B @ B.T
    shp = o.bc_shape(n)
    idx = list(np.ndindex(*shp))
    ref = np.array([[o.bc_exact_covariance(n, L, spec, bc, J, Jp) for Jp in idx] for J in idx])
    scale = np.abs(ref).max()
    np.testing.assert_allclose(Sig, ref, rtol=0, atol=1e-12 * scale)
    if bc == o.BC_NEUMANN:
        # the corner J = 0 has the periodic variance of the mirrored grid
        c0 = o.exact_covariance([2 * N for N in n], [2 * Li for Li in L], spec).flat[0]
        assert math.isclose(Sig[0, 0], c0, rel_tol=1e-12)


@pytest.mark.parametrize("n", [(16,), (8, 4), (4, 2, 8)])
def test_dirichlet_faces_are_exactly_zero(n):
    spec = o.Spectrum(family=o.MATERN, sigma=1.0, ell=0.2, nu=2.5)
    L = [1.0] * len(n)
    f = o.bc_field(n, L, spec, o.BC_DIRICHLET, 11)
    g = o.bc_field(n, L, spec, o.BC_NEUMANN, 11)
    for i in range(len(n)):
        assert np.all(np.take(f, 0, axis=i) == 0.0) and np.all(np.take(f, n[i], axis=i) == 0.0)
        assert np.abs(np.take(g, 0, axis=i)).max() > 0
    interior = f[tuple(slice(1, N) for N in n)]
    assert np.all(interior != 0.0)


def test_boundary_noise_moments():
    """a_K: mean 0 and variance 1 within 5 standard errors on 2^18 draws; seeds differ."""
    n = (511, 511)  # 512 x 512 points
    a = o.bc_normals(n, 3).ravel()
    m = a.size
    assert abs(a.mean()) < 5 / math.sqrt(m)
    assert abs(a.var() - 1.0) < 5 * math.sqrt(2.0 / m)
    # fourth moment of a normal is 3
    assert abs((a ** 4).mean() - 3.0) < 5 * math.sqrt(96.0 / m)
    b = o.bc_normals(n, 4).ravel()
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / math.sqrt(m)
    # neighbours (sharing a Philox call) are uncorrelated
    assert abs(np.mean(a[0::2] * a[1::2])) < 5 / math.sqrt(m / 2)


def test_boundary_lines_match_full_field():
    n = (8, 16)
    L = (1.0, 2.0)
    spec = o.Spectrum(family=o.MATERN, sigma=1.0, ell=0.2, nu=1.5)
    for bc in (o.BC_NEUMANN, o.BC_DIRICHLET):
        f = o.bc_field(n, L, spec, bc, 5)
        lines = o.bc_field_lines(n, L, spec, bc, 5, [(0,), (3,), (8,)])
        np.testing.assert_allclose(lines, f[[0, 3, 8]], rtol=0, atol=1e-12)
