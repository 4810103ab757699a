"""Seeded synthetic inputs shared by the tests and the benchmark: the shapes
and parameters of uneven batches.  Plain numpy random draws; no arithmetic of
the sampling method lives here."""
from __future__ import annotations

import numpy as np


def uneven_batch(count: int = 4096, seed: int = 0, frac_2d: float = 0.6, frac_1d: float = 0.3,
                 sides_2d=(32, 1024), lengths_1d=(2 ** 10, 2 ** 20), sides_3d=(32, 128),
                 ell=(0.005, 0.2), nu=(0.5, 3.0)):
    """Fields for one uneven batch: 60 % 2-D (each side a power of two drawn
    uniformly from sides_2d, non-square allowed), 30 % 1-D (length a power of
    two uniform in lengths_1d), 10 % 3-D (sides uniform in sides_3d); each with
    Matern sigma = 1 and (ell, nu) log-uniform.  Returns (shapes, lengths, specs)."""
    rng = np.random.default_rng(seed)

    def pow2_between(lo, hi, size=None):
        e = rng.integers(int(np.log2(lo)), int(np.log2(hi)) + 1, size=size)
        return 2 ** e

    shapes, lengths, specs = [], [], []
    for _ in range(count):
        u = rng.random()
        if u < frac_2d:
            shp = tuple(int(x) for x in pow2_between(*sides_2d, size=2))
        elif u < frac_2d + frac_1d:
            shp = (int(pow2_between(*lengths_1d)),)
        else:
            shp = tuple(int(x) for x in pow2_between(*sides_3d, size=3))
        shapes.append(shp)
        lengths.append((1.0,) * len(shp))
        specs.append(dict(family="matern", sigma=1.0,
                          ell=float(np.exp(rng.uniform(np.log(ell[0]), np.log(ell[1])))),
                          nu=float(np.exp(rng.uniform(np.log(nu[0]), np.log(nu[1]))))))
    return shapes, lengths, specs
