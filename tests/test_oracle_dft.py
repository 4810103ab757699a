"""Pins for the oracle's transforms against numpy's FFT (a library routine)."""
import numpy as np
import pytest

from oracle import grf_oracle as O


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8, 10, 12, 16, 32, 64, 128, 1024, 4096])
def test_fft_recursive_matches_library(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    np.testing.assert_allclose(O.fft_recursive(x, 1, -1), np.fft.fft(x, axis=1), rtol=0, atol=1e-12 * n)
    np.testing.assert_allclose(O.fft_recursive(x, 1, +1), n * np.fft.ifft(x, axis=1), rtol=0, atol=1e-12 * n)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 16])
def test_naive_dft_matches_library(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))
    np.testing.assert_allclose(O.dft_naive(x, 0, -1), np.fft.fft(x, axis=0), atol=1e-13 * max(n, 1))
    np.testing.assert_allclose(O.dft_naive(x, 0, +1), n * np.fft.ifft(x, axis=0), atol=1e-13 * max(n, 1))


@pytest.mark.parametrize("shape", [(8,), (4, 6), (8, 8), (4, 4, 4), (2, 8, 16)])
def test_dftn_matches_library(shape):
    rng = np.random.default_rng(len(shape))
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ntot = int(np.prod(shape))
    np.testing.assert_allclose(O.dftn(x, -1), np.fft.fftn(x), atol=1e-12 * ntot)
    np.testing.assert_allclose(O.dftn(x, +1), ntot * np.fft.ifftn(x), atol=1e-12 * ntot)
    np.testing.assert_allclose(O.dftn(x, +1, naive=True), ntot * np.fft.ifftn(x), atol=1e-12 * ntot)


def test_rfft_halfspectrum_matches_library():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((8, 16))
    np.testing.assert_allclose(O.rfft_halfspectrum(x), np.fft.rfftn(x), atol=1e-12)
