"""Uneven batches, in both modes (per-shape launches in one graph; one
persistent kernel): every field against the oracle, graph replay against the
plain launch, the two modes against each other, shard invariance, and the
bounded wait that turns a dependency that never resolves into GRF_ERR_TIMEOUT."""
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


def _api():
    from paper_1105_2737_gb300 import api
    return api


def _small_batch(count=36, seed=3):
    from paper_1105_2737_gb300.inputs import uneven_batch
    return uneven_batch(count, seed=seed, sides_2d=(32, 256), lengths_1d=(2 ** 10, 2 ** 16), sides_3d=(32, 64))


def _oracle_field(shape, L, spec, key):
    return O.alg2_field(shape, L, O.Spectrum(O.MATERN, spec["sigma"], spec["ell"], spec["nu"]), key)


@pytest.mark.parametrize("mode", ["shapes", "persistent"])
def test_every_field_matches_the_oracle(mode):
    shapes, lengths, specs = _small_batch()
    assert len({len(s) for s in shapes}) == 3  # 1-D, 2-D and 3-D all present
    b = _api().GRFBatch(shapes, lengths, specs, mode=mode)
    outs = b.sample(seed=500)
    torch.cuda.synchronize()
    assert b.status() == 0
    for i, (shp, L, sp) in enumerate(zip(shapes, lengths, specs)):
        ref = _oracle_field(shp, L, sp, 500 + i)
        got = outs[i].cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 2e-6 and np.abs(got - ref).max() <= 1e-5, (i, shp, rel)


@pytest.mark.parametrize("mode", ["shapes", "persistent"])
def test_graph_replay_equals_plain_launch(mode):
    shapes, lengths, specs = _small_batch(24, seed=4)
    b = _api().GRFBatch(shapes, lengths, specs, mode=mode)
    outs = b.empty()
    for seed in (10, 99, 10):
        b.sample(seed=seed, outs=outs)
        ref = [o.clone() for o in outs]
        for o in outs:
            o.zero_()
        b.sample(seed=seed, outs=outs, graph=True)
        b.sample(seed=seed, outs=outs, graph=True)  # a second replay of the same graph
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)
    assert b.status() == 0


def test_modes_draw_the_same_fields():
    """Per-shape launches and the persistent kernel: the same fields up to FP32 rounding."""
    shapes, lengths, specs = _small_batch(30, seed=8)
    a = _api().GRFBatch(shapes, lengths, specs, mode="shapes").sample(seed=77)
    p = _api().GRFBatch(shapes, lengths, specs, mode="persistent").sample(seed=77)
    torch.cuda.synchronize()
    for x, y in zip(a, p):
        x, y = x.double(), y.double()
        assert float((x - y).norm() / y.norm()) <= 2e-6 and float((x - y).abs().max()) <= 1e-5


def test_invalid_mode_is_rejected():
    from paper_1105_2737_gb300 import _lib as L
    shapes, lengths, specs = _small_batch(4, seed=9)
    b = _api().GRFBatch(shapes, lengths, specs)
    with pytest.raises(L.GRFError):
        L.grf_batch_set_mode(b.handle, 2)


def test_shard_invariance():
    """Fields are keyed by seed + index: two half batches with shifted seeds
    give the same fields as the whole batch."""
    shapes, lengths, specs = _small_batch(20, seed=5)
    api = _api()
    whole = api.GRFBatch(shapes, lengths, specs).sample(seed=1000)
    first = api.GRFBatch(shapes[:12], lengths[:12], specs[:12]).sample(seed=1000)
    second = api.GRFBatch(shapes[12:], lengths[12:], specs[12:]).sample(seed=1012)
    torch.cuda.synchronize()
    for a, b in zip(whole, first + second):
        assert torch.equal(a, b)


def test_withheld_dependency_times_out_and_context_survives():
    shapes, lengths, specs = _small_batch(12, seed=6)
    b = _api().GRFBatch(shapes, lengths, specs)
    outs = b.sample(seed=7)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    b.set_debug(withhold_field=0, timeout_ms=200.0)
    b.sample(seed=7, outs=outs)
    assert b.status() == 5  # GRF_ERR_TIMEOUT, reported, not a fault
    b.set_debug(-1)
    for o in outs:
        o.zero_()
    b.sample(seed=7, outs=outs)
    torch.cuda.synchronize()
    assert b.status() == 0
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)


def test_full_size_uneven_batch():
    """The 4096-field workload (60 % 2-D up to 1024^2, 30 % 1-D up to 2^20, 10 %
    3-D up to 128^3) in one launch; sampled fields checked against the oracle."""
    from paper_1105_2737_gb300.inputs import uneven_batch
    shapes, lengths, specs = uneven_batch(4096, seed=0)
    b = _api().GRFBatch(shapes, lengths, specs)
    outs = b.sample(seed=0)
    torch.cuda.synchronize()
    assert b.status() == 0
    picks = [i for i, s in enumerate(shapes) if np.prod(s) <= 2 ** 18][:6]
    picks += [max(range(len(shapes)), key=lambda i: np.prod(shapes[i]) if len(shapes[i]) == 1 else 0)]
    for i in picks:
        ref = _oracle_field(shapes[i], lengths[i], specs[i], i)
        got = outs[i].cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 2e-6 and np.abs(got - ref).max() <= 1e-5, (i, shapes[i], rel)
