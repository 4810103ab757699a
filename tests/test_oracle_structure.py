"""Pins for the index structure of §2 and the Hermitian arrangement of
Algorithm 2: the paper's Figure 1 and Figure 2 examples, the counts of the
appendix, and the vanishing imaginary part of the inverse transform."""
import math
import os
from itertools import product

import numpy as np
import pytest

from oracle import grf_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lines(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_fig1_self_conjugate_points():
    rows = _lines("fig1_grid4x4.txt")
    want = {(int(r[1]), int(r[2])) for r in rows if r[0] == "self"}
    assert set(O.self_conjugate_points((4, 4))) == want
    for r in rows:
        if r[0] == "pair":
            K, Lp = (int(r[1]), int(r[2])), (int(r[3]), int(r[4]))
            assert O.negate_index(K, (4, 4)) == Lp


@pytest.mark.parametrize("n", [(8,), (4, 4), (8, 6), (4, 4, 4), (2, 4, 6)])
def test_self_conjugate_count(n):
    assert len(O.self_conjugate_points(n)) == 2 ** len(n)


def _check_independent_set(pts, n):
    ntot = int(np.prod(n))
    d = len(n)
    assert len(pts) == (ntot + 2 ** d) // 2
    negs = {O.negate_index(K, n) for K in pts}
    # K and -K never both in the set unless K = -K; together they cover K^N
    for K in pts:
        if O.negate_index(K, n) != K:
            assert O.negate_index(K, n) not in pts
    assert pts | negs == set(np.ndindex(*n))


def test_fig2_independent_set_8x8():
    rows = _lines("fig2_LN_8x8.txt")
    n = tuple(int(v) for v in rows[0][1:])
    pts = set()
    for r in rows:
        if r[0] == "block":
            a, b, c, d = map(int, r[1:])
            pts |= set(product(range(a, b + 1), range(c, d + 1)))
    count = [int(r[1]) for r in rows if r[0] == "count"][0]
    assert len(pts) == count
    _check_independent_set(pts, n)


@pytest.mark.parametrize("n", [(8,), (8, 8), (4, 6), (4, 4, 4), (2, 4, 6), (6, 4, 2)])
def test_appendix_construction(n):
    _check_independent_set(O.independent_set_appendix(n), n)


@pytest.mark.parametrize("n", [(8,), (2,), (8, 8), (4, 6), (6, 2), (4, 4, 4), (2, 4, 6)])
def test_arrangement_loop_equals_vectorised(n):
    rng = np.random.default_rng(1)
    hs = O.half_shape(n)
    zr, zi = rng.standard_normal(hs), rng.standard_normal(hs)
    a = O.hermitian_arrangement(zr, zi, n)
    b = O.hermitian_arrangement_vectorised(zr, zi, n)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("n", [(8,), (8, 8), (4, 6), (4, 4, 4), (2, 4, 6)])
def test_arrangement_is_hermitian_and_uses_LN_degrees(n):
    rng = np.random.default_rng(2)
    hs = O.half_shape(n)
    zr, zi = rng.standard_normal(hs), rng.standard_normal(hs)
    xi = O.hermitian_arrangement_vectorised(zr, zi, n)
    full = O.extend_hermitian(xi, n)
    for K in np.ndindex(*n):
        assert full[K] == np.conj(full[O.negate_index(K, n)])
    # self-conjugate entries are the plain real normal (scale factor 1, not 2^-1/2)
    for K in O.self_conjugate_points(n):
        assert full[K] == zr[K] if K[-1] <= n[-1] // 2 else True
    # the number of real degrees of freedom actually used is N_tot: each point
    # of H that carries its own fresh value contributes 2 (1 if self-conjugate)
    used = 0
    for K in np.ndindex(*hs):
        if O.is_self_conjugate(K, n):
            used += 1
        elif xi[K] == (zr[K] + 1j * zi[K]) / math.sqrt(2):
            used += 2
    assert used == int(np.prod(n))


@pytest.mark.parametrize("n,L", [((64, 64), (1.0, 1.0)), ((32, 16), (2.0, 0.5)), ((16,), (1.0,)), ((8, 8, 8), (1, 1, 1))])
@pytest.mark.parametrize("alg", [1, 2])
def test_imaginary_part_vanishes(n, L, alg):
    spec = O.Spectrum(O.MATERN, 1.0, 0.1, 1.5)
    fc = O.alg2_field(n, L, spec, 3, return_complex=True) if alg == 2 else O.alg1_field(n, L, spec, 3, return_complex=True)
    s = O.sqrt_scale(n, L, spec)
    bound = 64 * np.finfo(np.float64).eps * float(np.abs(s).sum()) * 6.0
    assert np.abs(fc.imag).max() <= bound
    assert np.abs(fc.real).max() > 1e-3


def test_field_lines_equal_full_field():
    n, L = (16, 12, 8), (1.0, 1.0, 2.0)
    spec = O.Spectrum(O.GAUSSIAN, 1.0, 0.1, 0.0)
    f = O.alg2_field(n, L, spec, 11)
    AH = O.alg2_halfspectrum(n, L, spec, 11)
    picks = [(0, 0), (3, 5), (15, 11)]
    lines = O.field_lines(AH, n, picks)
    for J, ln in zip(picks, lines):
        np.testing.assert_allclose(ln, f[J], atol=1e-12)
