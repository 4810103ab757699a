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
