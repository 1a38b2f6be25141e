"""Host-side logic of bench.py: the roofline traffic read from the ncu summary
is scaled to the launch's algorithmic bytes and withdrawn as soon as a kernel
source it was measured on changes; the workload table names every config."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_scales_the_measured_ratio_and_tracks_the_sources(tmp_path, monkeypatch):
    root = tmp_path
    (root / "profiles").mkdir()
    (root / "k").mkdir()
    src = root / "k" / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (root / "profiles" / "traffic.json").write_text(json.dumps(
        {"ts_inner": {"dram_per_algorithmic_byte": 0.9, "sources": ["k/kernel.cu"], "sha256": sha}}))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert abs(bench.traffic_for("ts_inner", 1000.0) - 900.0) < 1e-9
    assert bench.traffic_for("spmv", 1000.0) is None
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.traffic_for("ts_inner", 1000.0) is None


def test_committed_traffic_summary_matches_the_kernel_sources():
    """The committed capture still describes the committed kernels (else the
    bench reports traffic null until the capture is repeated)."""
    import pytest
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    ent = d["ts_inner"]
    assert 0.5 < ent["dram_per_algorithmic_byte"] < 1.5
    h = hashlib.sha256()
    for f in ent["sources"]:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest() != ent["sha256"]:
        pytest.skip("kernel sources changed since the ncu capture: the bench reports traffic null")


def test_workload_table():
    assert set(bench.WORKLOADS) == {"diffusion128", "q1pencil96", "chunglu22", "aniso128"}
    for key, w in bench.WORKLOADS.items():
        assert w["p"] <= w["k"] < w["q"] <= 64 and w["l"] >= 0 and w["tol"] == 1e-8, key
    assert bench.WORKLOAD["key"] == "diffusion128"
