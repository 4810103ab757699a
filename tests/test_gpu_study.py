"""The Monte Carlo covariance estimator of the paper's 1-D study (§4),
Cov(x_j) = (1/count) sum_b eta_b(0) eta_b(x_j): the CUDA sums against the
oracle's fields on the same seeds, and the estimate against the exact
covariance of the grid within Monte Carlo bands."""
import numpy as np
import pytest

from oracle import grf_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the paper's 1-D example: gamma(p) = 32e6/pi (100 + p^2)^-4 in angular
# frequency on [-pi, pi], i.e. Matern nu = 7/2, ell = 1/10 in cycles on L = 2 pi
SPEC = O.Spectrum(O.MATERN, 1.0, 0.1, 3.5)
L = 2 * np.pi


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_2737_gb300 import build
    build()


def _plan(N, max_batch):
    from paper_1105_2737_gb300 import api
    return api.GRF((N,), (L,), family="matern", sigma=1.0, ell=0.1, nu=3.5, max_batch=max_batch)


@pytest.mark.parametrize("N,count,max_batch", [(8, 100, 128), (32, 50, 16), (4096, 24, 8), (16384, 5, 4)])
def test_cov_origin_sums_match_the_oracle(N, count, max_batch):
    """Chunked (count > max_batch) and unchunked; the 1-D row path and the
    four-step path (N = 16384)."""
    g = _plan(N, max_batch)
    got = g.cov_origin(seed=77, count=count).cpu().numpy()
    f = O.sample((N,), (L,), SPEC, 77, count)
    ref = (f[:, :1] * f).sum(axis=0)
    # the sums are bilinear in the fields, whose points carry at most 1e-5 sigma
    # of FP32 error (sigma = 1): |d(f0 fj)| <= 1e-5 (|f0| + |fj|) per sample
    bound = 1e-5 * (np.abs(f[:, :1]) + np.abs(f)).sum(axis=0)
    assert np.all(np.abs(got - ref) <= bound), (np.abs(got - ref) / bound).max()


def test_cov_origin_sums_accumulate_across_calls():
    g = _plan(16, 64)
    s = g.cov_origin(seed=5, count=40)
    s = g.cov_origin(seed=45, count=40, sums=s)
    whole = g.cov_origin(seed=5, count=80)
    np.testing.assert_allclose(s.cpu().numpy(), whole.cpu().numpy(), rtol=1e-12, atol=1e-12)


def test_cov_origin_within_monte_carlo_bands():
    """2^21 samples on 16 points: the estimate lies within 5 standard
    deviations sqrt((c(0)^2 + c(x_j)^2) / count) of the exact covariance of
    the grid, c(x_j) = (1/|D|) sum_K S(p_K) cos(2 pi K j / N)."""
    N, count = 16, 1 << 21
    g = _plan(N, 1 << 15)
    cov = g.cov_origin(seed=1000, count=count).cpu().numpy() / count
    c = O.exact_covariance((N,), (L,), SPEC)
    band = 5 * np.sqrt((c[0] ** 2 + c ** 2) / count)
    assert np.all(np.abs(cov - c) <= band), (np.abs(cov - c) / band).max()


# the four cases of the paper's Fig. 3 (2-D polynomial family of §4),
# gamma(p) = (m^(k l) + (p_1^(2k) + p_2^(2k))^l)^(-n), as (m, n, k, l)
FIG3 = [(10.0, 1, 1, 2), (0.75, 1, 1, 2), (10.0, 3, 1, 1), (5.0, 1, 3, 1)]


@pytest.mark.parametrize("m,n,k,l", FIG3)
def test_paper_family_point_covariance(m, n, k, l):
    """§4's statistical test of the 2-D family: the covariance of the grid point
    x_0 with every other grid point over 2^17 fields (64^2 points on [0, 8]^2)
    lies within 5.5 standard deviations sqrt((c(0)^2 + c(x_j)^2) / count) of the
    exact covariance of the grid at all 4096 points, negative lobes included."""
    from paper_1105_2737_gb300 import api
    N, Lb, count = 64, 8.0, 1 << 17
    g = api.GRF((N, N), (Lb, Lb), family="paper_poly", sigma=1.0, m=m, k=k, l=l, n=n, max_batch=8192)
    cov = g.cov_origin(seed=4242, count=count).cpu().numpy() / count
    exact = O.exact_covariance((N, N), (Lb, Lb), O.Spectrum(O.PAPER_POLY, 1.0, m=m, k=k, l=l, n=n))
    band = 5.5 * np.sqrt((exact[0, 0] ** 2 + exact ** 2) / count)
    assert cov.shape == (N, N)
    assert np.all(np.abs(cov - exact) <= band), (np.abs(cov - exact) / band).max()
    g.close()


def test_boundary_field_corner_covariance():
    """The estimator on a Neumann field: covariance of the corner with every
    point over 2^17 fields against the method-of-images covariance."""
    from paper_1105_2737_gb300 import api
    n, Lb, count = (16, 16), (1.0, 1.0), 1 << 17
    g = api.GRFBoundary(n, Lb, bc="neumann", family="matern", sigma=1.0, ell=0.1, nu=1.5, max_batch=8192)
    cov = g.cov_origin(seed=99, count=count).cpu().numpy() / count
    spec = O.Spectrum(O.MATERN, 1.0, 0.1, 1.5)
    exact = np.array([[O.bc_exact_covariance(n, Lb, spec, O.BC_NEUMANN, (0, 0), (a, b)) for b in range(17)]
                      for a in range(17)])
    band = 5.5 * np.sqrt((exact[0, 0] ** 2 + exact ** 2) / count)
    assert np.all(np.abs(cov - exact) <= band), (np.abs(cov - exact) / band).max()
    g.close()
