"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeds, element by element.  FP32 fields: relative L2 <= 2e-6 and max abs
<= 1e-5 sigma; FP64 plain form: <= 1e-12 relative; Philox words bit-exact."""
import numpy as np
import pytest

from oracle import grf_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_L2 = 2e-6
MAX_ABS = 1e-5  # times sigma


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_2737_gb300 import build
    build()


def _api():
    from paper_1105_2737_gb300 import api
    return api


FAM = {"matern": O.MATERN, "gaussian": O.GAUSSIAN, "paper_poly": O.PAPER_POLY}


def _ospec(family, **kw):
    base = dict(sigma=1.0, ell=0.1, nu=1.5, m=1.0, k=1, l=1, n=1, normalize_discrete=0)
    base.update(kw)
    return O.Spectrum(FAM[family], base["sigma"], base["ell"], base["nu"], base["m"], base["k"], base["l"],
                      base["n"], base["normalize_discrete"])


def _compare(got, ref, sigma=1.0, rel=REL_L2, mx=MAX_ABS):
    got = np.asarray(got, dtype=np.float64)
    e_rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    e_max = np.abs(got - ref).max()
    assert e_rel <= rel and e_max <= mx * sigma, (e_rel, e_max)
    return e_rel, e_max


def test_philox_words_bit_exact():
    from paper_1105_2737_gb300 import _lib as L
    for key, tag, q0 in [(0, 0, 0), (1, 1, 2**32 - 5), (2**64 - 1, 0, 2**40), (0xDEADBEEFCAFEF00D, 2, 12345)]:
        cnt = 4096
        out = torch.empty(4 * cnt, dtype=torch.int32, device="cuda")
        L.grf_philox_words(key, tag, q0, cnt, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32).reshape(cnt, 4)
        q = np.arange(q0, q0 + cnt, dtype=np.uint64)
        want = np.stack(O.philox_words(q, tag, key), axis=1)
        np.testing.assert_array_equal(got, want)


CASES_2D = [((64, 64), (1.0, 1.0), "matern", dict(ell=0.1, nu=1.5), 2),
            ((256, 128), (2.0, 1.0), "matern", dict(ell=0.05, nu=0.5, sigma=1.7), 3),
            ((128, 512), (1.0, 1.0), "gaussian", dict(ell=0.03), 2),
            ((8, 8), (1.0, 1.0), "matern", dict(ell=0.2, nu=2.5), 3),
            ((2, 2), (1.0, 1.0), "matern", dict(ell=0.3, nu=1.0), 2),
            ((4, 16), (1.0, 3.0), "gaussian", dict(ell=0.2), 2),
            ((32, 2), (1.0, 1.0), "matern", dict(ell=0.2, nu=1.5), 2),
            ((1024, 32), (1.0, 1.0), "matern", dict(ell=0.01, nu=2.5), 2),
            ((16, 8192), (1.0, 1.0), "matern", dict(ell=0.05, nu=1.5), 1),
            ((64, 64), (1.0, 1.0), "paper_poly", dict(m=10.0, k=1, l=2, n=1, sigma=1.0), 1),
            ((32, 64), (1.0, 1.0), "matern", dict(ell=0.1, nu=1.5, normalize_discrete=1), 1)]


@pytest.mark.parametrize("alg", [2, 1])
@pytest.mark.parametrize("case", range(len(CASES_2D)))
def test_fields_2d(case, alg):
    n, Lb, fam, kw, batch = CASES_2D[case]
    g = _api().GRF(n, Lb, family=fam, alg=alg, max_batch=batch, **kw)
    f = g.sample(seed=11, batch=batch).cpu().numpy()
    ref = O.sample(n, Lb, _ospec(fam, **kw), seed=11, batch=batch, alg=alg)
    _compare(f, ref, sigma=np.sqrt((ref ** 2).mean()))


CASES_1D = [(2, 1.0), (4, 1.0), (16, 1.0), (64, 2.0), (1024, 1.0), (8192, 1.0)]


@pytest.mark.parametrize("alg", [2, 1])
@pytest.mark.parametrize("N,Lx", CASES_1D)
def test_fields_1d(N, Lx, alg):
    kw = dict(ell=0.05, nu=1.5)
    g = _api().GRF((N,), (Lx,), family="matern", alg=alg, max_batch=5, **kw)
    f = g.sample(seed=3, batch=5).cpu().numpy()
    ref = O.sample((N,), (Lx,), _ospec("matern", **kw), seed=3, batch=5, alg=alg)
    _compare(f, ref)


CASES_3D = [((16, 16, 16), (1.0, 1.0, 1.0), "gaussian", dict(ell=0.1)),
            ((8, 32, 64), (1.0, 2.0, 1.0), "matern", dict(ell=0.1, nu=1.5)),
            ((32, 32, 32), (1.0, 1.0, 1.0), "gaussian", dict(ell=0.03)),
            ((2, 4, 2), (1.0, 1.0, 1.0), "matern", dict(ell=0.3, nu=0.7)),
            ((64, 16, 128), (1.0, 1.0, 1.0), "matern", dict(ell=0.05, nu=2.5))]


@pytest.mark.parametrize("alg", [2, 1])
@pytest.mark.parametrize("case", range(len(CASES_3D)))
def test_fields_3d(case, alg):
    n, Lb, fam, kw = CASES_3D[case]
    g = _api().GRF(n, Lb, family=fam, alg=alg, max_batch=2, **kw)
    f = g.sample(seed=5, batch=2).cpu().numpy()
    ref = O.sample(n, Lb, _ospec(fam, **kw), seed=5, batch=2, alg=alg)
    _compare(f, ref)


@pytest.mark.parametrize("n", [(64, 64), (16,), (8, 8, 8), (32, 16)])
@pytest.mark.parametrize("alg", [2, 1])
def test_fp64_plain_form(n, alg):
    kw = dict(ell=0.1, nu=1.5)
    Lb = (1.0,) * len(n)
    g = _api().GRF(n, Lb, family="matern", alg=alg, precision="fp64", max_batch=2, **kw)
    f = g.sample(seed=1, batch=2).cpu().numpy()
    ref = O.sample(n, Lb, _ospec("matern", **kw), seed=1, batch=2, alg=alg)
    e = np.linalg.norm(f - ref) / np.linalg.norm(ref)
    assert e <= 1e-12, e


def test_same_seed_same_fields_and_batch_split():
    g = _api().GRF((128, 64), (1.0, 1.0), ell=0.05, nu=1.5, max_batch=8)
    a = g.sample(seed=100, batch=8).clone()
    b = g.sample(seed=100, batch=8)
    assert torch.equal(a, b)
    c = g.sample(seed=104, batch=4)
    assert torch.equal(a[4:], c)  # field b of seed s is field b - k of seed s + k


def test_sample_host_matches_device():
    g = _api().GRF((256, 256), (1.0, 1.0), ell=0.05, nu=1.5, max_batch=6)
    a = g.sample(seed=9, batch=6).cpu()
    h = g.sample_host(seed=9, batch=6)
    assert torch.equal(a, h)


@pytest.mark.parametrize("n", [(64, 32), (128,), (16, 8, 32)])
def test_rfft_forward(n):
    g = _api().GRF(n, (1.0,) * len(n), ell=0.1, nu=1.5, max_batch=3)
    x = torch.randn((3,) + n, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    X = g.rfft(x).cpu().numpy()
    ref = np.stack([O.rfft_halfspectrum(x[i].cpu().numpy().astype(np.float64)) for i in range(3)])
    e = np.linalg.norm(X - ref) / np.linalg.norm(ref)
    assert e <= 2e-6, e


@pytest.mark.parametrize("n", [(64, 64), (256,), (16, 32, 8)])
@pytest.mark.parametrize("fam", ["matern", "gaussian"])
def test_adjoint_matches_oracle(n, fam):
    kw = dict(ell=0.08, nu=1.5, sigma=1.3)
    Lb = (1.0,) * len(n)
    g = _api().GRF(n, Lb, family=fam, max_batch=3, **kw)
    G = torch.randn((3,) + n, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    gp = g.backward(21, G).cpu().numpy()
    ref = O.adjoint_grad(n, Lb, _ospec(fam, **kw), 21, G.cpu().numpy().astype(np.float64))
    scale = np.abs(ref).max(axis=0)
    scale[scale == 0] = 1.0
    assert np.all(np.abs(gp - ref) <= 1e-4 * scale + 1e-12), (gp, ref)


def test_noise_recovery():
    """DFT(f) / (N_tot s_K) recovers xi_K exactly in exact arithmetic (Eq. drf)."""
    n, Lb = (64, 32), (1.0, 1.0)
    spec = _ospec("matern", ell=0.1, nu=1.5)
    g = _api().GRF(n, Lb, family="matern", ell=0.1, nu=1.5, max_batch=1)
    f = g.sample(seed=77, batch=1)[0].cpu().numpy().astype(np.float64)
    F = O.rfft_halfspectrum(f)
    s = O.sqrt_scale(n, Lb, spec, half=True)
    xi = F / (64 * 32 * s)
    ref = O.alg2_noise(n, 77)
    assert np.abs(xi - ref).max() <= 2e-5


def test_same_noise_two_spectra():
    """Figures 4-6 of §4 reuse one white noise with several densities: the
    half spectra of two such fields differ mode by mode by s1/s2."""
    n, Lb = (128, 128), (1.0, 1.0)
    g1 = _api().GRF(n, Lb, family="matern", ell=0.05, nu=0.5, max_batch=1)
    g2 = _api().GRF(n, Lb, family="matern", ell=0.05, nu=2.5, max_batch=1)
    F1 = g1.rfft(g1.sample(seed=3)).cpu().numpy()[0]
    F2 = g2.rfft(g2.sample(seed=3)).cpu().numpy()[0]
    s1 = O.sqrt_scale(n, Lb, _ospec("matern", ell=0.05, nu=0.5), half=True)
    s2 = O.sqrt_scale(n, Lb, _ospec("matern", ell=0.05, nu=2.5), half=True)
    big = np.abs(F2) > 1e-3 * np.abs(F2).max()
    ratio = (F1 / np.where(big, F2, 1))[big]
    np.testing.assert_allclose(ratio, (s1 / s2)[big], rtol=1e-3)


def test_invalid_calls_raise():
    api = _api()
    from paper_1105_2737_gb300._lib import GRFError
    g = api.GRF((32, 32), (1.0, 1.0), max_batch=2)
    with pytest.raises(GRFError):
        g.sample(seed=0, batch=3)
    with pytest.raises(GRFError):
        api.GRF((24, 32), (1.0, 1.0))
    g64 = api.GRF((32, 32), (1.0, 1.0), precision="fp64")
    with pytest.raises(GRFError):
        g64.backward(0, torch.zeros((1, 32, 32), dtype=torch.float64, device="cuda"))
