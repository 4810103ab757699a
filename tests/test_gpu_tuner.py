"""Schedules: every radix (4, 8, 16 points per thread) and tile choice gives
the oracle's fields, schedules stored in the tuning cache are applied by
grf_plan_create, and grf_plan_tune picks a valid schedule."""
import os

import numpy as np
import pytest

from oracle import grf_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_2737_gb300 import build
    build()


def _key2(shape, alg, max_batch):
    n = list(shape) + [1] * (3 - len(shape))
    gpu = torch.cuda.get_device_name().replace(" ", "_")
    return "plan|%s|%d" % (gpu, len(shape)) + "".join("x%d" % v for v in n) + "|alg%d|b%d" % (alg, max_batch)


# (T, colA.P, colA.C, colB.P, colB.C, row.P, row.C, pipe[, row_tma])
SCHEDS_2D = [(1, 16, 1, 16, 1, 16, 1, 1), (8, 8, 2, 16, 1, 8, 4, 1), (4, 4, 4, 16, 1, 4, 8, 2),
             (16, 16, 4, 16, 1, 16, 2, 4), (2, 8, 1, 16, 1, 4, 1, 1),
             # c2r pass fed by bulk copies: tile T = C, T < C, T = 1, pipelined
             (2, 16, 1, 16, 1, 16, 2, 1, 1), (4, 8, 2, 16, 1, 8, 8, 1, 1), (1, 16, 1, 16, 1, 4, 4, 1, 1),
             (16, 16, 4, 16, 1, 16, 16, 2, 1), (8, 16, 2, 16, 1, 16, 8, 4, 1),
             # 256-thread radix-16 geometries (C N = 4096): the compile-time forms of
             # the noise pass (N_1 = 256, 16 column pairs) and the c2r pass (M = 256, 16 rows)
             (2, 16, 16, 16, 1, 16, 16, 1, 0), (16, 16, 16, 16, 1, 16, 16, 1, 0)]


@pytest.mark.parametrize("sched", SCHEDS_2D)
def test_forced_schedules_2d(sched, tmp_path):
    from paper_1105_2737_gb300 import api
    shape, Lb, batch = (256, 512), (1.0, 1.0), 3
    path = tmp_path / "tune.txt"
    path.write_text(_key2(shape, 2, batch) + " " + " ".join(str(v) for v in sched) + "\n")
    os.environ["GRF_TUNE_CACHE"] = str(path)
    try:
        g = api.GRF(shape, Lb, ell=0.05, nu=1.5, max_batch=batch)
    finally:
        del os.environ["GRF_TUNE_CACHE"]
    sch = g.schedule
    assert (sch["T"], sch["colA_P"], sch["colA_C"], sch["row_P"], sch["row_C"], sch["pipe"]) == \
        (sched[0], sched[1], sched[2], sched[5], sched[6], sched[7])
    assert sch["row_tma"] == (sched[8] if len(sched) > 8 else 0)
    f = g.sample(seed=4, batch=batch).cpu().numpy()
    ref = O.sample(shape, Lb, O.Spectrum(O.MATERN, 1.0, 0.05, 1.5), 4, batch)
    rel = np.linalg.norm(f - ref) / np.linalg.norm(ref)
    assert rel <= 2e-6 and np.abs(f - ref).max() <= 1e-5, rel


@pytest.mark.parametrize("sched", [(1, 8, 4, 4, 8, 8, 4, 1), (1, 4, 2, 8, 2, 16, 4, 2),
                                   (1, 8, 4, 4, 8, 16, 4, 1, 1), (1, 16, 1, 16, 1, 8, 8, 2, 1)])
def test_forced_schedules_3d(sched, tmp_path):
    from paper_1105_2737_gb300 import api
    shape, Lb, batch = (32, 64, 64), (1.0, 1.0, 1.0), 2
    path = tmp_path / "tune.txt"
    path.write_text(_key2(shape, 2, batch) + " " + " ".join(str(v) for v in sched) + "\n")
    os.environ["GRF_TUNE_CACHE"] = str(path)
    try:
        g = api.GRF(shape, Lb, family="gaussian", ell=0.05, max_batch=batch)
    finally:
        del os.environ["GRF_TUNE_CACHE"]
    sch = g.schedule
    assert (sch["colA_P"], sch["colB_P"], sch["row_P"]) == (sched[1], sched[3], sched[5])
    f = g.sample(seed=6, batch=batch).cpu().numpy()
    ref = O.sample(shape, Lb, O.Spectrum(O.GAUSSIAN, 1.0, 0.05, 0.0), 6, batch)
    rel = np.linalg.norm(f - ref) / np.linalg.norm(ref)
    assert rel <= 2e-6, rel


def test_tune_picks_a_valid_schedule(tmp_path):
    from paper_1105_2737_gb300 import api
    os.environ["GRF_TUNE_CACHE"] = str(tmp_path / "tune.txt")
    try:
        g = api.GRF((512, 512), (1.0, 1.0), ell=0.05, nu=2.5, max_batch=16)
        sch = g.tune()
        assert sch["colA_P"] in (4, 8, 16) and sch["row_P"] in (4, 8, 16) and sch["T"] in (1, 2, 4, 8, 16)
        text = (tmp_path / "tune.txt").read_text()
        assert "plan|" in text
        # a new plan with the same key picks the stored schedule up
        g2 = api.GRF((512, 512), (1.0, 1.0), ell=0.05, nu=2.5, max_batch=16)
        assert g2.schedule == sch
    finally:
        del os.environ["GRF_TUNE_CACHE"]
    f = g2.sample(seed=1, batch=2).cpu().numpy()
    ref = O.sample((512, 512), (1.0, 1.0), O.Spectrum(O.MATERN, 1.0, 0.05, 2.5), 1, 2)
    assert np.linalg.norm(f - ref) / np.linalg.norm(ref) <= 2e-6


def test_bulk_copy_c2r_falls_back_below_one_group(tmp_path):
    """A bulk-copy schedule whose row group (C = 8 rows) is larger than the rows
    of the call (one 4 x 8 field: 4 rows) runs the plain row kernel instead and
    still gives the oracle's field; the full batch takes the bulk-copy kernel."""
    from paper_1105_2737_gb300 import api
    shape, Lb = (4, 8), (1.0, 1.0)
    sched = (4, 4, 1, 16, 1, 4, 8, 1, 1)
    path = tmp_path / "tune.txt"
    path.write_text(_key2(shape, 2, 2) + " " + " ".join(str(v) for v in sched) + "\n")
    os.environ["GRF_TUNE_CACHE"] = str(path)
    try:
        g = api.GRF(shape, Lb, ell=0.2, nu=1.5, max_batch=2)
    finally:
        del os.environ["GRF_TUNE_CACHE"]
    assert g.schedule["row_tma"] == 1 and g.schedule["row_C"] == 8
    spec = O.Spectrum(O.MATERN, 1.0, 0.2, 1.5)
    for batch in (1, 2):
        f = g.sample(seed=9, batch=batch).cpu().numpy()
        ref = O.sample(shape, Lb, spec, 9, batch)
        assert np.abs(f - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_tune_keeps_a_cached_schedule(tmp_path):
    """A plan whose schedule came from the tuning cache keeps it when tuned
    again (no re-timing), unless GRF_TUNE_FORCE=1."""
    from paper_1105_2737_gb300 import api
    shape, Lb, batch = (256, 512), (1.0, 1.0), 3
    sched = (8, 8, 2, 16, 1, 8, 4, 1)
    path = tmp_path / "tune.txt"
    path.write_text(_key2(shape, 2, batch) + " " + " ".join(str(v) for v in sched) + "\n")
    os.environ["GRF_TUNE_CACHE"] = str(path)
    try:
        g = api.GRF(shape, Lb, ell=0.05, nu=1.5, max_batch=batch)
        before = dict(g.schedule)
        after = g.tune()
        assert after == before and (after["T"], after["colA_P"], after["row_C"]) == (8, 8, 4)
        assert path.read_text().count("\n") == 1  # nothing re-timed or stored
    finally:
        del os.environ["GRF_TUNE_CACHE"]


def test_forced_compile_time_geometries_3d(tmp_path):
    """3-D schedule whose noise pass (N_1 = 256, 16 columns) and c2r pass
    (M = 128, 32 rows) take the compile-time forms, with the axis-2 pair pass
    at 16 points (N_2 = 16, general form): fields match the oracle."""
    from paper_1105_2737_gb300 import api
    shape, Lb, batch = (256, 16, 256), (1.0, 1.0, 1.0), 2
    sched = (1, 16, 16, 16, 16, 16, 32, 1, 0)
    path = tmp_path / "tune.txt"
    path.write_text(_key2(shape, 2, batch) + " " + " ".join(str(v) for v in sched) + "\n")
    os.environ["GRF_TUNE_CACHE"] = str(path)
    try:
        g = api.GRF(shape, Lb, ell=0.05, nu=1.5, max_batch=batch)
    finally:
        del os.environ["GRF_TUNE_CACHE"]
    sch = g.schedule
    assert (sch["colA_P"], sch["colA_C"], sch["row_P"], sch["row_C"]) == (16, 16, 16, 32)
    f = g.sample(seed=13, batch=batch).cpu().numpy()
    ref = O.sample(shape, Lb, O.Spectrum(O.MATERN, 1.0, 0.05, 1.5), 13, batch)
    rel = np.linalg.norm(f - ref) / np.linalg.norm(ref)
    assert rel <= 2e-6 and np.abs(f - ref).max() <= 1e-5 * np.sqrt((ref ** 2).mean()), rel


def test_full_size_in_the_bench_schedule(tmp_path):
    """4096^2 x 64 in the schedule the tuner picks for the bench on GB300
    (T = 4, one column pair and two rows per CTA, radix 16, the compile-time
    forms): sampled rows of field 0 and the whole of field 63 against the oracle."""
    from paper_1105_2737_gb300 import api
    shape, Lb, batch = (4096, 4096), (1.0, 1.0), 64
    path = tmp_path / "tune.txt"
    path.write_text(_key2(shape, 2, batch) + " 4 16 1 16 1 16 2 1 0\n")
    os.environ["GRF_TUNE_CACHE"] = str(path)
    try:
        g = api.GRF(shape, Lb, ell=0.05, nu=2.5, max_batch=batch)
    finally:
        del os.environ["GRF_TUNE_CACHE"]
    sch = g.schedule
    assert (sch["T"], sch["colA_P"], sch["colA_C"], sch["row_P"], sch["row_C"]) == (4, 16, 1, 16, 2)
    f = g.sample(seed=640, batch=batch)
    spec = O.Spectrum(O.MATERN, 1.0, 0.05, 2.5)
    rows = [(0,), (3,), (2048,), (4095,)]
    ref = O.field_lines(O.alg2_halfspectrum(shape, Lb, spec, 640), shape, rows)
    got = np.stack([f[(0,) + J].cpu().numpy() for J in rows]).astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 2e-6 and np.abs(got - ref).max() <= 1e-5, rel
    # the last field of the call, whole
    ref = O.alg2_field(shape, Lb, spec, 640 + 63)
    got = f[63].cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 2e-6 and np.abs(got - ref).max() <= 1e-5, rel
    g.close()
