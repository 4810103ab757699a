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


@pytest.mark.parametrize("N", [2 ** 14, 2 ** 16, 2 ** 17, 2 ** 20])
def test_fields_1d_four_step(N):
    """Long 1-D grids: c2r by the four-step decomposition M = A B."""
    kw = dict(ell=0.01, nu=1.5)
    batch = 3
    g = _api().GRF((N,), (1.0,), family="matern", max_batch=batch, **kw)
    f = g.sample(seed=8, batch=batch).cpu().numpy()
    ref = O.sample((N,), (1.0,), _ospec("matern", **kw), seed=8, batch=batch)
    _compare(f, ref)


def test_fields_1d_four_step_fp64():
    kw = dict(ell=0.01, nu=1.5)
    g = _api().GRF((2 ** 16,), (1.0,), family="matern", precision="fp64", max_batch=2, **kw)
    f = g.sample(seed=8, batch=2).cpu().numpy()
    ref = O.sample((2 ** 16,), (1.0,), _ospec("matern", **kw), seed=8, batch=2)
    assert np.linalg.norm(f - ref) / np.linalg.norm(ref) <= 1e-12


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


# sizes whose odd part is 3, 5 or 7 (the FP64 plain form's radix-3/5/7 stages);
# Lb anisotropic, Gaussian and paper families too
MIXED = [((6,), "matern"), ((10,), "gaussian"), ((14,), "matern"), ((30,), "paper_poly"), ((1000,), "matern"),
         ((12, 20), "matern"), ((96, 80), "gaussian"), ((6, 10, 14), "matern"), ((2, 42, 6), "paper_poly"),
         ((3000,), "matern")]


@pytest.mark.parametrize("case", range(len(MIXED)))
@pytest.mark.parametrize("alg", [2, 1])
def test_fp64_mixed_radix_sizes(case, alg):
    n, fam = MIXED[case]
    kw = dict(ell=0.1, nu=1.5) if fam != "paper_poly" else dict(m=2.0, k=1, l=2, n=1)
    Lb = tuple(1.0 + 0.25 * i for i in range(len(n)))
    g = _api().GRF(n, Lb, family=fam, alg=alg, precision="fp64", max_batch=2, **kw)
    f = g.sample(seed=3, batch=2).cpu().numpy()
    ref = O.sample(n, Lb, _ospec(fam, **kw), seed=3, batch=2, alg=alg)
    e = np.linalg.norm(f - ref) / np.linalg.norm(ref)
    assert e <= 1e-12, e
    assert np.abs(f - ref).max() <= 1e-12 * np.abs(ref).max() * 10


@pytest.mark.parametrize("case", range(len(MIXED)))
@pytest.mark.parametrize("alg", [2, 1])
def test_fp32_mixed_radix_sizes(case, alg):
    """FP32 plans off powers of two (the FP32 plain form) within the FP32 bar."""
    n, fam = MIXED[case]
    kw = dict(ell=0.1, nu=1.5) if fam != "paper_poly" else dict(m=2.0, k=1, l=2, n=1)
    Lb = tuple(1.0 + 0.25 * i for i in range(len(n)))
    g = _api().GRF(n, Lb, family=fam, alg=alg, precision="fp32", max_batch=2, **kw)
    f = g.sample(seed=3, batch=2).cpu().numpy()
    ref = O.sample(n, Lb, _ospec(fam, **kw), seed=3, batch=2, alg=alg)
    _compare(f, ref, sigma=1.0 if fam != "paper_poly" else float(np.sqrt((ref ** 2).mean())))


def test_fp32_mixed_radix_full_size_3000sq():
    """3000^2 (2^3 3 5^3) FP32, batch 2 in one call: the whole second field
    against the oracle (the bench's 3000^2 workload)."""
    kw = dict(ell=0.05, nu=2.5)
    g = _api().GRF((3000, 3000), (1.0, 1.0), family="matern", precision="fp32", max_batch=2, **kw)
    f = g.sample(seed=40, batch=2)[1].cpu().numpy()
    ref = O.alg2_field((3000, 3000), (1.0, 1.0), _ospec("matern", **kw), 41)
    _compare(f, ref)
    g.close()


# FP32 2-D Algorithm 2 off powers of two: the fused mixed-radix passes.  Cases
# with several column CTAs and a ragged last one ((M + 1) mod C1 != 0), radix 7
# on either axis, a power-of-two axis beside a mixed one, N1 = 2, and the
# largest last axis (M = 4096).
FUSED = [((2, 6), "matern"), ((1000, 210), "matern"), ((448, 252), "gaussian"), ((14, 8192), "matern"),
         ((4096, 3000), "matern"), ((3000, 4096), "paper_poly"), ((96, 80), "matern"), ((6, 2), "matern")]


@pytest.mark.parametrize("case", range(len(FUSED)))
def test_fp32_mixed_fused_passes(case):
    """The fields of a batch of 3 against the oracle (the last one alone on the
    12 M-point grids); the plan runs the two
    fused passes per call (timing records), not the per-field plain form."""
    from paper_1105_2737_gb300 import _lib as L
    n, fam = FUSED[case]
    kw = dict(ell=0.05, nu=1.5) if fam != "paper_poly" else dict(m=2.0, k=1, l=2, n=1)
    Lb = (1.0, 1.5)
    g = _api().GRF(n, Lb, family=fam, precision="fp32", max_batch=3, **kw)
    L.grf_plan_timing(g.handle, 16)
    f = g.sample(seed=77, batch=3).cpu().numpy()
    _, recs = L.grf_plan_timing_read(g.handle)
    L.grf_plan_timing(g.handle, 0)
    kinds = [k for k, _ in recs]
    if n[1] // 2 > 1:  # the fused schedule needs M >= 2
        assert kinds == ["noise_columns", "rows_c2r"], kinds
    else:
        assert set(kinds) == {"plain64"}, kinds
    sig = None
    for b in (range(3) if n[0] * n[1] < 4_000_000 else (2,)):  # the oracle takes ~10 s per 12 M-point field
        ref = O.alg2_field(n, Lb, _ospec(fam, **kw), 77 + b)
        if fam == "paper_poly":
            sig = float(np.sqrt((ref ** 2).mean()))
        _compare(f[b], ref, sigma=1.0 if sig is None else sig)
    g.close()


def test_fp32_mixed_fused_host_delivery_and_plain_form():
    """The fused mixed-radix passes: grf_sample_host gives the device fields bit
    for bit, a call of 2 fields on a plan of 5 gives the first 2 of a call of 5,
    and the plain form of the same plan (GRF_MIXED_FUSED=0) agrees within the
    FP32 bar (both are checked against the oracle elsewhere)."""
    import os
    n = (600, 350)  # 2^3 3 5^2 x 2 5^2 7: radices 3, 5, 5, 8 and 5, 5, 7
    kw = dict(ell=0.04, nu=1.5)
    g = _api().GRF(n, (1.0, 1.0), family="matern", precision="fp32", max_batch=5, **kw)
    d5 = g.sample(seed=21, batch=5).cpu().numpy()
    d2 = g.sample(seed=21, batch=2).cpu().numpy()
    h = g.sample_host(seed=21, batch=5).numpy()
    assert np.array_equal(d5, h)
    assert np.array_equal(d5[:2], d2)
    g.close()
    os.environ["GRF_MIXED_FUSED"] = "0"
    try:
        gp = _api().GRF(n, (1.0, 1.0), family="matern", precision="fp32", max_batch=5, **kw)
        p5 = gp.sample(seed=21, batch=5).cpu().numpy()
        gp.close()
    finally:
        del os.environ["GRF_MIXED_FUSED"]
    e = np.linalg.norm(p5 - d5) / np.linalg.norm(d5)
    assert e <= 2 * REL_L2, e


def test_fp32_mixed_plan_has_no_adjoint_or_rfft():
    from paper_1105_2737_gb300 import _lib as L
    g = _api().GRF((12, 20), (1.0, 1.0), precision="fp32", max_batch=1)
    with pytest.raises(L.GRFError):
        g.backward(0, torch.zeros((1, 12, 20), device="cuda"))
    with pytest.raises(L.GRFError):
        g.rfft(torch.zeros((1, 12, 20), device="cuda"))


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
    """DFT(f) = N_tot s_K xi_K (Eq. drf with the unnormalised inverse DFT): the
    forward transform of a GPU field recovers the oracle's noise."""
    n, Lb = (64, 32), (1.0, 1.0)
    spec = _ospec("matern", ell=0.1, nu=1.5)
    g = _api().GRF(n, Lb, family="matern", ell=0.1, nu=1.5, max_batch=1)
    f = g.sample(seed=77, batch=1)[0].cpu().numpy().astype(np.float64)
    F = O.rfft_halfspectrum(f)
    s = O.sqrt_scale(n, Lb, spec, half=True)
    ref = O.alg2_noise(n, 77)
    ntot = 64 * 32
    # the identity over every mode, against the size of the spectrum
    assert np.abs(F - ntot * s * ref).max() <= 1e-6 * ntot * np.abs(s * ref).max()
    # and xi itself wherever s_K is not tiny (FP32 error / s_K grows at high k)
    big = s >= 1e-2 * s.max()
    assert np.abs(F / (ntot * s) - ref)[big].max() <= 2e-5


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
        api.GRF((22, 32), (1.0, 1.0))  # prime factor 11
    g64 = api.GRF((32, 32), (1.0, 1.0), precision="fp64")
    with pytest.raises(GRFError):
        g64.backward(0, torch.zeros((1, 32, 32), dtype=torch.float64, device="cuda"))


def test_monte_carlo_covariance_bands():
    """Sample covariance of many GPU fields at several lags within 5 standard
    deviations of the exact covariance c(r) (Isserlis variance of the estimator)."""
    n, Lb = (32, 32), (1.0, 1.0)
    spec = _ospec("matern", ell=0.1, nu=1.5)
    c = O.exact_covariance(n, Lb, spec)
    for alg in (2, 1):
        Mf = 20000
        g = _api().GRF(n, Lb, family="matern", ell=0.1, nu=1.5, alg=alg, max_batch=Mf)
        f = g.sample(seed=123456, batch=Mf).double()
        for r in [(0, 0), (1, 0), (0, 3), (5, 7), (16, 16)]:
            est = float((f * torch.roll(f, shifts=(-r[0], -r[1]), dims=(1, 2))).mean())
            cp = np.roll(c, shift=(-r[0], -r[1]), axis=(0, 1))
            cm = np.roll(c, shift=(r[0], r[1]), axis=(0, 1))
            var = float((c ** 2 + cp * cm).sum()) / (Mf * 32 * 32)
            assert abs(est - c[r]) <= 5 * np.sqrt(var), (alg, r, est, c[r])


def _sampled_rows(n, Lb, spec, seed, fields, rows):
    """Oracle rows f[b, j1, :] (2-D) or lines f[b, j1, j2, :] (3-D) by the definition."""
    out = {}
    for b in fields:
        AH = O.alg2_halfspectrum(n, Lb, spec, seed + b)
        out[b] = O.field_lines(AH, n, rows)
    return out


@pytest.mark.parametrize("shape,fam,kw,batch,fields,rows", [
    ((4096, 4096), "matern", dict(ell=0.05, nu=2.5), 64, [0, 37, 63], [(0,), (1,), (2047,), (2048,), (4095,)]),
    ((4096, 4096), "matern", dict(ell=0.01, nu=0.5), 64, [5], [(0,), (3000,)]),
    # rough and short-range: s_K decays slowly, so an error with a nonzero mean
    # over the modes adds up coherently at points like (0, 0)
    ((4096, 4096), "matern", dict(ell=0.002, nu=0.5), 64, [3], [(0,), (777,)]),
    ((512, 512), "matern", dict(ell=0.05, nu=0.5), 64, [0, 63], [(0,), (255,), (511,)]),
    ((256, 256, 256), "gaussian", dict(ell=0.03), 8, [0, 7], [(0, 0), (128, 5), (255, 255)]),
])
def test_full_size_sampled_rows(shape, fam, kw, batch, fields, rows):
    """The configurations the bench times, at full size and batch, in the same
    launch configuration: sampled rows against the oracle's rows."""
    Lb = (1.0,) * len(shape)
    g = _api().GRF(shape, Lb, family=fam, max_batch=batch, **kw)
    f = g.sample(seed=0, batch=batch)
    ref = _sampled_rows(shape, Lb, _ospec(fam, **kw), 0, fields, rows)
    for b in fields:
        got = np.stack([f[(b,) + tuple(J)].cpu().numpy() for J in rows])
        _compare(got, ref[b])
    # the whole batch has the variance of this grid, c(0) = (1/|D|) sum_K S(p_K)
    # (a cheap check on every field; the spread is the batch's sampling error)
    var = float((f.double() ** 2).mean())
    c0 = float(O.scaled_density(shape, Lb, _ospec(fam, **kw)).sum())
    assert 0.7 * c0 < var < 1.4 * c0, (var, c0)


def test_autograd_power_spectrum_loss():
    """Differentiation config: 1024^2 x 16 Matern (ell = 0.05, nu = 1.5); loss = L2
    mismatch of the radially binned power spectrum (64 bins) against a target
    (ell = 0.08, nu = 2.0).  The gradient through the autograd.Function (the
    adjoint kernel) matches the oracle's analytic gradient."""
    api = _api()
    n, Lb, B = (1024, 1024), (1.0, 1.0), 16
    g = api.GRF(n, Lb, family="matern", sigma=1.0, ell=0.05, nu=1.5, max_batch=B)
    loss_spec = O.BinnedLossSpec(nbins=64, target=O.Spectrum(O.MATERN, 1.0, 0.08, 2.0))
    bins = torch.as_tensor(O.radial_bins(n, Lb, 64), device="cuda")
    w = torch.as_tensor(O.half_weights(n), device="cuda")
    T, Wb = O.binned_power(O.scaled_density(n, Lb, loss_spec.target, half=True), O.radial_bins(n, Lb, 64),
                           O.half_weights(n), 64)
    T = torch.as_tensor(T, device="cuda")
    Wb = torch.as_tensor(np.where(Wb > 0, Wb, 1.0), device="cuda")
    m = bins >= 0
    theta = torch.tensor([1.0, 0.05, 1.5], dtype=torch.float64, requires_grad=True)
    f = api.grf_fields(theta, g, 0, B)
    F = torch.fft.rfft2(f.double())  # the user's loss (not part of the library)
    P = (F.real ** 2 + F.imag ** 2) / (1024 * 1024) ** 2
    Pb = torch.zeros((B, 64), dtype=torch.float64, device="cuda")
    Pb.index_add_(1, bins[m], (P * w)[:, m])
    Pb = Pb / Wb
    loss = ((Pb - T) ** 2).sum() / B
    loss.backward()
    Lref, gref = O.power_loss_and_grad(n, Lb, O.Spectrum(O.MATERN, 1.0, 0.05, 1.5), 0, B, loss_spec)
    assert abs(float(loss.detach()) - Lref) <= 1e-4 * abs(Lref)
    np.testing.assert_allclose(theta.grad.numpy(), gref, rtol=1e-4, atol=1e-8 * np.abs(gref).max())
