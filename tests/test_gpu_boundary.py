"""GPU parity of the Neumann / Dirichlet fields (cosine / sine transform
variant of the method) through the C ABI, against the FP64 oracle on the same
seeds: element by element at small sizes that span several CTAs and ragged
line counts, sampled lines at 4096^2 and 128^3, exact zeros on Dirichlet
faces, and the image-sum variance over many fields."""
import numpy as np
import pytest

from oracle import grf_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_L2 = 2e-6
MAX_ABS = 1e-5  # times sigma

FAM = {"matern": O.MATERN, "gaussian": O.GAUSSIAN, "paper_poly": O.PAPER_POLY}
BC = {"neumann": O.BC_NEUMANN, "dirichlet": O.BC_DIRICHLET}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_2737_gb300 import build
    build()


def _api():
    from paper_1105_2737_gb300 import api
    return api


def _ospec(family, **kw):
    base = dict(sigma=1.0, ell=0.1, nu=1.5, m=1.0, k=1, l=1, n=1)
    base.update(kw)
    return O.Spectrum(FAM[family], base["sigma"], base["ell"], base["nu"], base["m"], base["k"], base["l"],
                      base["n"], 0)


def _compare(got, ref, sigma=1.0):
    got = np.asarray(got, dtype=np.float64)
    e_rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    e_max = np.abs(got - ref).max()
    assert e_rel <= REL_L2 and e_max <= MAX_ABS * sigma, (e_rel, e_max)
    return e_rel, e_max


# (intervals, lengths, family, params, batch): every FFT length from 4 to 8192,
# line counts that leave the last CTA of a pass partly empty, 1-D to 3-D
CASES = [
    ((2,), (1.0,), "matern", dict(ell=0.3, nu=1.5), 5),
    ((4,), (1.0,), "gaussian", dict(ell=0.2), 3),
    ((8,), (2.0,), "matern", dict(ell=0.2, nu=0.5), 7),
    ((64,), (1.0,), "paper_poly", dict(m=2.0, k=1, l=2, n=1), 3),
    ((4096,), (1.0,), "matern", dict(ell=0.01, nu=2.5), 3),
    ((16, 32), (1.0, 2.0), "matern", dict(ell=0.1, nu=1.5), 2),
    ((64, 8), (1.5, 0.5), "gaussian", dict(ell=0.07), 3),
    ((2, 128), (1.0, 1.0), "matern", dict(ell=0.2, nu=2.5), 2),
    ((256, 256), (1.0, 1.0), "paper_poly", dict(m=4.0, k=2, l=1, n=2), 1),
    ((8, 16, 4), (1.0, 0.5, 2.0), "matern", dict(ell=0.2, nu=1.5), 2),
    ((32, 32, 32), (1.0, 1.0, 1.0), "gaussian", dict(ell=0.1), 1),
    # the fixed geometries 2N = 1024, 2048, 4096 (rows and strided launches)
    ((512, 1024), (1.0, 1.0), "matern", dict(ell=0.05, nu=1.5), 2),
    ((2048, 64), (2.0, 1.0), "gaussian", dict(ell=0.05), 2),
    ((2048, 4, 512), (1.0, 0.5, 1.0), "matern", dict(ell=0.1, nu=2.5), 1),
]


@pytest.mark.parametrize("bc", ["neumann", "dirichlet"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_boundary_field_parity(case, bc):
    n, L, fam, kw, batch = CASES[case]
    g = _api().GRFBoundary(n, L, bc=bc, family=fam, max_batch=batch, **kw)
    seed = 1000 + 17 * case
    out = g.sample(seed, batch)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    spec = _ospec(fam, **kw)
    for b in range(batch):
        ref = O.bc_field(n, L, spec, BC[bc], seed + b)
        _compare(got[b], ref)
        if bc == "dirichlet":
            for i in range(len(n)):
                assert np.all(np.take(got[b], 0, axis=i) == 0.0)
                assert np.all(np.take(got[b], n[i], axis=i) == 0.0)
    g.close()


@pytest.mark.parametrize("bc", ["neumann", "dirichlet"])
def test_boundary_full_size_2d_lines(bc):
    """4096^2 intervals (4097^2 points), batch 2 as one call; sampled lines of field 1."""
    n, L = (4096, 4096), (1.0, 1.0)
    kw = dict(ell=0.02, nu=2.5)
    g = _api().GRFBoundary(n, L, bc=bc, family="matern", max_batch=2, **kw)
    out = g.sample(77, 2)
    rows = [0, 1, 2047, 4095, 4096]
    torch.cuda.synchronize()
    got = out[1, rows].cpu().numpy()
    ref = O.bc_field_lines(n, L, _ospec("matern", **kw), BC[bc], 78, [(r,) for r in rows])
    _compare(got, ref)
    g.close()


def test_boundary_full_size_3d_lines():
    n, L = (128, 128, 128), (1.0, 2.0, 1.0)
    kw = dict(ell=0.05)
    g = _api().GRFBoundary(n, L, bc="neumann", family="gaussian", max_batch=1, **kw)
    out = g.sample(5, 1)
    lines = [(0, 0), (3, 64), (128, 127), (77, 128)]
    torch.cuda.synchronize()
    got = np.stack([out[0, a, b].cpu().numpy() for a, b in lines])
    ref = O.bc_field_lines(n, L, _ospec("gaussian", **kw), O.BC_NEUMANN, 5, lines)
    _compare(got, ref)
    g.close()


@pytest.mark.parametrize("bc", ["neumann", "dirichlet"])
def test_boundary_variance_is_image_sum(bc):
    """Pointwise variance over 2^15 fields against 1/2 (c(0) +- c(2 x_j)) of the
    mirrored grid, within 6 standard errors (the variance of a variance
    estimate of a normal is 2 v^2 / count)."""
    n, L = (32,), (1.0,)
    kw = dict(ell=0.1, nu=1.5)
    count = 1 << 15
    g = _api().GRFBoundary(n, L, bc=bc, family="matern", max_batch=count, **kw)
    f = g.sample(9, count).double()
    var = (f * f).mean(dim=0).cpu().numpy()
    spec = _ospec("matern", **kw)
    want = np.array([O.bc_exact_covariance(n, L, spec, BC[bc], (j,), (j,)) for j in range(n[0] + 1)])
    band = 6 * np.sqrt(2.0 / count) * want + 1e-12
    assert np.all(np.abs(var - want) <= band), np.max(np.abs(var - want) / band)
    g.close()


def test_boundary_set_spectrum_and_host_delivery():
    """grf_plan_set_spectrum rebuilds c_K (fields equal a fresh plan's, bit for
    bit); grf_sample_host delivers the same fields as grf_sample."""
    api = _api()
    n, L = (64, 32), (1.0, 0.5)
    g = api.GRFBoundary(n, L, bc="dirichlet", family="matern", ell=0.1, nu=1.5, max_batch=3)
    g.set_params("matern", sigma=1.3, ell=0.05, nu=2.5)
    a = g.sample(11, 3)
    fresh = api.GRFBoundary(n, L, bc="dirichlet", family="matern", sigma=1.3, ell=0.05, nu=2.5, max_batch=3)
    b = fresh.sample(11, 3)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    h = g.sample_host(11, 3)
    assert torch.equal(h, a.cpu())
    ref = O.bc_field(n, L, _ospec("matern", sigma=1.3, ell=0.05, nu=2.5), O.BC_DIRICHLET, 12)
    _compare(h[1].numpy(), ref, sigma=1.3)
    from paper_1105_2737_gb300 import _lib as Lb
    with pytest.raises(Lb.GRFError):
        g.set_params("gaussian", ell=0.1)  # the family is fixed at creation
    g.close()
    fresh.close()
