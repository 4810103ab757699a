"""The 3-D plane path (pass 1: noise, axis 1 and the first radix-R step of
axis 2; pass 2: one sub-plane per CTA, staged by a bulk copy, the rest of axis
2 and the c2r rows, rows written by bulk copies) against the FP64 oracle, for
every split R of axis 2 it takes (1, 2, 4), transform lengths N1 = 8..1024 (below
256 pass 1 is the ordinary column pass writing whole planes with padded rows),
both forms of pass 2 (two slots per persistent CTA, one slot per CTA), ragged
k3 groups (M + 1 is odd), several fields per launch and plans the path does not
take; and against the three-pass form (GRF_PLANE3=0) on the same seeds."""
import os

import numpy as np
import pytest

from oracle import grf_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_L2 = 2e-6
MAX_ABS = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_2737_gb300 import build
    build()


def _api():
    from paper_1105_2737_gb300 import api
    return api


def _plane_radix(g):
    from paper_1105_2737_gb300 import _lib as L
    return L.grf_plan_query(g.handle, 17)


def _check(got, ref, what):
    got = np.asarray(got, dtype=np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    mx = np.abs(got - ref).max()
    assert rel <= REL_L2 and mx <= MAX_ABS, (what, rel, mx)


# shape, the split R the plan must take (0: the three-pass form), batch, spectrum
CASES = [((256, 16, 256), 1, 2, O.Spectrum(O.MATERN, 1.0, 0.05, 1.5)),
         ((256, 256, 128), 2, 1, O.Spectrum(O.GAUSSIAN, 1.0, 0.03)),
         ((256, 256, 256), 4, 2, O.Spectrum(O.MATERN, 1.0, 0.02, 0.5)),
         ((256, 256, 512), 4, 1, O.Spectrum(O.MATERN, 1.0, 0.05, 2.5)),   # one slot, 512 threads
         ((512, 256, 64), 2, 2, O.Spectrum(O.MATERN, 1.3, 0.05, 1.5)),
         ((1024, 64, 128), 1, 2, O.Spectrum(O.MATERN, 1.0, 0.1, 1.5)),
         ((128, 128, 128), 1, 2, O.Spectrum(O.GAUSSIAN, 1.0, 0.03)),      # pass 1: the column pass, padded rows
         ((8, 32, 64), 1, 3, O.Spectrum(O.MATERN, 1.0, 0.1, 1.5)),
         ((64, 16, 128), 1, 2, O.Spectrum(O.MATERN, 1.0, 0.05, 2.5)),
         ((512, 512, 512), 0, 1, O.Spectrum(O.GAUSSIAN, 1.0, 0.03)),      # runs of 4 k3 need R <= 2
         ((2048, 16, 32), 0, 3, O.Spectrum(O.MATERN, 1.0, 0.05, 1.5))]

FAM = {O.MATERN: "matern", O.GAUSSIAN: "gaussian"}


@pytest.mark.parametrize("case", range(len(CASES)))
def test_plane_path_against_the_oracle(case):
    shape, R, batch, sp = CASES[case]
    Lb = (1.0, 1.5, 1.0)
    g = _api().GRF(shape, Lb, family=FAM[sp.family], sigma=sp.sigma, ell=sp.ell, nu=sp.nu, max_batch=batch)
    assert _plane_radix(g) == R
    seed = 31 * case + 7
    f = g.sample(seed=seed, batch=batch)
    npts = int(np.prod(shape))
    for b in sorted({0, batch - 1}):
        if npts <= 1 << 21:  # whole fields
            ref = O.alg2_field(shape, Lb, sp, seed + b)
            _check(f[b].cpu().numpy(), ref, (shape, b))
        else:  # lines f[j1, j2, :], spread over j1, both residues of j2 mod R
            n1, n2 = shape[0], shape[1]
            lines = [(0, 0), (1, 1), (n1 // 2, n2 - 1), (n1 - 1, n2 // 2 + 1), (n1 // 3, 5)]
            ref = O.field_lines(O.alg2_halfspectrum(shape, Lb, sp, seed + b), shape, lines)
            got = np.stack([f[(b,) + J].cpu().numpy() for J in lines])
            _check(got, ref, (shape, b))
    from paper_1105_2737_gb300 import _lib as L
    assert L.grf_status_word(g.handle, torch.cuda.current_stream().cuda_stream) == 0
    g.close()


def test_plane_path_equals_three_pass_form():
    """Same seeds through the plane path and the three-pass form: the same
    fields within the FP32 bar (both are FP32 evaluations of one sum)."""
    shape, Lb = (256, 256, 256), (1.0, 1.0, 1.0)
    kw = dict(family="gaussian", sigma=1.0, ell=0.03, max_batch=2)
    a = _api().GRF(shape, Lb, **kw)
    assert _plane_radix(a) == 4
    fa = a.sample(seed=100, batch=2).double()
    os.environ["GRF_PLANE3"] = "0"
    try:
        b = _api().GRF(shape, Lb, **kw)
    finally:
        del os.environ["GRF_PLANE3"]
    assert _plane_radix(b) == 0
    fb = b.sample(seed=100, batch=2).double()
    rel = float(torch.linalg.vector_norm(fa - fb) / torch.linalg.vector_norm(fb))
    assert rel <= REL_L2 and float((fa - fb).abs().max()) <= MAX_ABS, rel
    a.close()
    b.close()


def test_plane_path_host_delivery_and_reuse():
    """grf_sample_host and back-to-back calls of one plan give the device fields."""
    g = _api().GRF((256, 32, 128), (1.0, 1.0, 1.0), family="matern", ell=0.05, nu=1.5, max_batch=3)
    assert _plane_radix(g) >= 1
    a = g.sample(seed=9, batch=3).cpu()
    g.sample(seed=1000, batch=3)
    h = g.sample_host(seed=9, batch=3)
    assert torch.equal(a, h)
    g.close()
