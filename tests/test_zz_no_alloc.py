"""The allocation-free 2-D entry point, grf_sample_2d_static, for callers that
cannot allocate device memory when they sample (an application that owns all
of the device's memory, or a loop where cudaMalloc / cudaFree would
synchronise the device).  It must draw the same fields as grf_sample on an
ordinary plan.  Collected last: a failure here leaves every other test run."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_2737_gb300 import build
    build()
    from paper_1105_2737_gb300 import _lib
    return _lib


def _reference(L, n, Lb, spec, seed, batch):
    """The same fields through a plan (grf_plan_create + grf_sample)."""
    h = L.grf_plan_create(2, n, Lb, spec, L.GRF_ALG_ONE_FFT, L.GRF_FP32, batch)
    try:
        out = torch.empty((batch,) + tuple(n), dtype=torch.float32, device="cuda")
        L.grf_sample(h, seed, batch, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        L.grf_plan_destroy(h)


def _static(L, n, Lb, spec, seed, batch):
    out = torch.empty((batch,) + tuple(n), dtype=torch.float32, device="cuda")
    L.grf_sample_2d_static(n, Lb, spec, seed, batch, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_two_calls_in_a_row_match_the_plan_path(L):
    calls = [((256, 512), (1.0, 2.0), L.make_spectrum(L.GRF_MATERN, 1.0, 0.05, 1.5), 7, 3),
             ((1024, 64), (1.0, 1.0), L.make_spectrum(L.GRF_GAUSSIAN, 1.3, 0.02, 0.0), 1234, 2)]
    got = [_static(L, *c) for c in calls]  # back to back: the second reuses the scratch array
    for c, g in zip(calls, got):
        ref = _reference(L, *c)
        rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        assert rel <= 2e-6 and np.abs(g - ref).max() <= 1e-5, (c[0], rel)


def test_worst_case_smallest_grids_and_paper_family(L):
    """The largest grid the array holds (1024 x 1024, two fields in a row), the
    smallest grids (2 x 4 and 4 x 2: one row of the c2r pass, trimmed CTAs) and
    the polynomial family of the paper, each against the plan path."""
    calls = [((1024, 1024), (1.0, 1.0), L.make_spectrum(L.GRF_MATERN, 1.0, 0.02, 2.5), 99, 2),
             ((2, 4), (1.0, 1.0), L.make_spectrum(L.GRF_MATERN, 1.0, 0.3, 1.5), 5, 3),
             ((4, 2), (1.0, 2.0), L.make_spectrum(L.GRF_GAUSSIAN, 1.0, 0.3, 0.0), 6, 3),
             ((64, 128), (8.0, 8.0), L.make_spectrum(L.GRF_PAPER_POLY, 1.0, 0.0, 0.0, 10.0, 1, 2, 1), 17, 2)]
    for c in calls:
        g = _static(L, *c)
        ref = _reference(L, *c)
        rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        scale = max(1.0, float(np.sqrt((ref ** 2).mean())))
        assert rel <= 2e-6 and np.abs(g - ref).max() <= 1e-5 * scale, (c[0], rel)


def test_against_the_oracle(L):
    """Every field of a call against the FP64 oracle directly (not only the
    plan path): a Matern and a paper-family grid, within the FP32 bar."""
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle import grf_oracle as O
    calls = [((256, 128), (1.0, 2.0), L.make_spectrum(L.GRF_MATERN, 1.0, 0.05, 1.5),
              O.Spectrum(O.MATERN, 1.0, 0.05, 1.5), 41, 2),
             ((64, 128), (8.0, 8.0), L.make_spectrum(L.GRF_PAPER_POLY, 1.0, 0.0, 0.0, 10.0, 1, 2, 1),
              O.Spectrum(O.PAPER_POLY, 1.0, 0.0, 0.0, 10.0, 1, 2, 1), 17, 2)]
    for n, Lb, spec, ospec, seed, batch in calls:
        g = _static(L, n, Lb, spec, seed, batch)
        for b in range(batch):
            ref = O.alg2_field(n, Lb, ospec, seed + b)
            rel = np.linalg.norm(g[b] - ref) / np.linalg.norm(ref)
            scale = max(1.0, float(np.sqrt((ref ** 2).mean())))
            assert rel <= 2e-6 and np.abs(g[b] - ref).max() <= 1e-5 * scale, (n, b, rel)


def test_sizes_beyond_the_scratch_are_rejected(L):
    out = torch.empty(4, dtype=torch.float32, device="cuda")
    nn = (C.c_int64 * 2)(2048, 64)
    LL = (C.c_double * 2)(1.0, 1.0)
    sp = L.make_spectrum()
    st = L.lib().grf_sample_2d_static(nn, LL, C.byref(sp), 0, 1, C.c_void_p(out.data_ptr()), None)
    assert st == L.GRF_ERR_INVALID_ARG
    assert b"1024" in L.lib().grf_last_error()
