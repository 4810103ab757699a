"""Pins for the oracle's gradients: digamma against scipy, d log S against
finite differences, the analytic loss gradient and the adjoint against FP64
central finite differences (h = 1e-6) of the oracle's own forward pipeline."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import grf_oracle as O


@pytest.mark.parametrize("x", [0.25, 0.5, 1.0, 1.5, 2.0, 3.5, 7.0, 40.0])
def test_digamma(x):
    assert abs(O.digamma(x) - special.digamma(x)) < 1e-13 * max(1, abs(special.digamma(x)))


@pytest.mark.parametrize("fam", [O.MATERN, O.GAUSSIAN])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_dlogS_matches_finite_differences(fam, d):
    n = (8,) * d
    L = (1.0,) * d
    base = dict(family=fam, sigma=1.2, ell=0.15, nu=1.7)
    ds = O.dlogS(n, L, O.Spectrum(**base))
    h = 1e-6
    for t, name in enumerate(["sigma", "ell", "nu"]):
        if fam == O.GAUSSIAN and name == "nu":
            continue
        up = dict(base); up[name] += h
        dn = dict(base); dn[name] -= h
        pu = O.spectral_density(O.frequency_grid(n, L, half=True), O.Spectrum(**up))
        pd = O.spectral_density(O.frequency_grid(n, L, half=True), O.Spectrum(**dn))
        fd = (np.log(pu) - np.log(pd)) / (2 * h)
        np.testing.assert_allclose(ds[t], fd, rtol=1e-7, atol=1e-7)


def test_power_identity_and_loss_value():
    n, L = (16, 12), (1.0, 1.0)
    spec = O.Spectrum(O.MATERN, 1.0, 0.1, 1.5)
    f = O.alg2_field(n, L, spec, 4)
    F = O.dftn(f, -1)[..., : n[-1] // 2 + 1]
    A = O.alg2_halfspectrum(n, L, spec, 4)
    np.testing.assert_allclose(np.abs(F) ** 2 / (16 * 12) ** 2, np.abs(A) ** 2, atol=1e-14)
    loss = O.BinnedLossSpec(nbins=8)
    Lv, _ = O.power_loss_and_grad(n, L, spec, 4, 2, loss)
    Lf = O.power_loss_from_fields(O.sample(n, L, spec, 4, 2), n, L, loss)
    assert abs(Lv - Lf) <= 1e-12 * max(1.0, abs(Lf))


@pytest.mark.parametrize("n,L", [((32, 32), (1.0, 1.0)), ((64,), (1.0,)), ((8, 8, 16), (1.0, 1.0, 2.0))])
def test_loss_gradient_matches_finite_differences(n, L):
    base = dict(family=O.MATERN, sigma=1.0, ell=0.05 if len(n) < 3 else 0.2, nu=1.5)
    loss = O.BinnedLossSpec(nbins=16)
    _, g = O.power_loss_and_grad(n, L, O.Spectrum(**base), 0, 2, loss)
    h = 1e-6
    for t, name in enumerate(["sigma", "ell", "nu"]):
        up = dict(base); up[name] += h
        dn = dict(base); dn[name] -= h
        fu = O.power_loss_from_fields(O.sample(n, L, O.Spectrum(**up), 0, 2), n, L, loss)
        fd_ = O.power_loss_from_fields(O.sample(n, L, O.Spectrum(**dn), 0, 2), n, L, loss)
        fd = (fu - fd_) / (2 * h)
        assert abs(fd - g[t]) <= 1e-6 * max(abs(g).max(), 1e-12) + 1e-9 * abs(g[t]), (name, fd, g[t])


@pytest.mark.parametrize("fam", [O.MATERN, O.GAUSSIAN])
def test_adjoint_matches_finite_differences(fam):
    n, L = (16, 8), (1.0, 0.5)
    base = dict(family=fam, sigma=0.9, ell=0.1, nu=2.5)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((2,) + n)
    g = O.adjoint_grad(n, L, O.Spectrum(**base), 7, G)
    h = 1e-6
    for t, name in enumerate(["sigma", "ell", "nu"]):
        if fam == O.GAUSSIAN and name == "nu":
            assert np.all(g[:, t] == 0)
            continue
        up = dict(base); up[name] += h
        dn = dict(base); dn[name] -= h
        fu = O.sample(n, L, O.Spectrum(**up), 7, 2)
        fdn = O.sample(n, L, O.Spectrum(**dn), 7, 2)
        fd = ((fu - fdn) * G).sum(axis=(1, 2)) / (2 * h)
        np.testing.assert_allclose(g[:, t], fd, rtol=1e-7, atol=1e-9)
