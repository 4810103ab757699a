"""The JSON-line contract of bench.py's reference arm (the FP64 oracle timed on
the host cores), checked on the CPU: one line with the metric, the timing keys,
the oracle as cpu_baseline and an e2e object without host-device copies."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT,
                       env=dict(os.environ, GRF_ORACLE_WORKERS="2"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_kernel_fingerprints_cover_each_kernels_sources():
    """The traffic figure of a kernel stays valid while the sources it is built
    from are unchanged: the fingerprint covers the kernel's .cu files, the
    launch code and every header they include, and nothing else."""
    import importlib
    B = importlib.import_module("paper_1105_2737_gb300.build")
    noise = B._include_closure(B.KERNEL_SOURCES["noise_columns"])
    rows = B._include_closure(B.KERNEL_SOURCES["rows_c2r"])
    for f in ("noise_fast.cu", "noise_fast.cuh", "common.cuh", "fft_core.cuh", "bodies.cuh", "api.cu", "grf.h"):
        assert f in noise, f
    for f in ("spec_other.cu", "c2r_tma.cu", "tma.cuh", "fft_core.cuh", "api.cu"):
        assert f in rows, f
    for f in ("r2r.cuh", "r2r.cu", "mixed_fused.cu", "plane3d.cu", "batch.cu"):
        assert f not in noise and f not in rows, f
    fp = {k: B.kernel_fingerprint(k) for k in B.KERNEL_SOURCES}
    assert all(len(v) == 64 for v in fp.values()) and fp["noise_columns"] != fp["rows_c2r"]
