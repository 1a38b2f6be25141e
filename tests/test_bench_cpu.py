"""Host-side logic of bench.py: the roofline traffic read from the ncu summary
is scaled to the launch's algorithmic bytes and withdrawn as soon as a kernel
source it was measured on changes; eigenvalue errors against the stored
oracle runs; the workload table names every config."""
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
        {"diffusion128/ts_inner": {"dram_per_algorithmic_byte": 0.9, "sources": ["k/kernel.cu"], "sha256": sha}}))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert abs(bench.traffic_for("diffusion128", "ts_inner", 1000.0) - 900.0) < 1e-9
    assert bench.traffic_for("chunglu22", "ts_inner", 1000.0) is None
    assert bench.traffic_for("diffusion128", "spmv", 1000.0) is None
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.traffic_for("diffusion128", "ts_inner", 1000.0) is None


def test_committed_traffic_summaries_are_well_formed():
    """Every committed capture names its sources and a plausible DRAM ratio;
    one whose sources changed since is reported null by the bench."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return
    for key, ent in json.load(open(path)).items():
        assert "/" in key, key
        assert 0.3 < ent["dram_per_algorithmic_byte"] < 3.0, key
        assert ent["sources"] and all(os.path.exists(os.path.join(ROOT, f)) for f in ent["sources"]), key
        assert len(ent["sha256"]) == 64, key


def test_eig_error_against_a_stored_run():
    ref = {"evals": [1.0, 2.0, 4.0], "status": "ok"}
    assert abs(bench.eig_error([1.0, 2.0 + 2e-9, 4.0], ref) - 1e-9) < 1e-15
    assert bench.eig_error([1.0], None) is None
    stored = bench.stored_oracle_run("chunglu22")
    assert stored is not None and len(stored["evals"]) == 16


def test_workload_table():
    assert set(bench.WORKLOADS) == {"diffusion128", "q1pencil96", "chunglu22", "chunglu20", "aniso128"}
    for key, w in bench.WORKLOADS.items():
        assert w["p"] <= w["k"] < w["q"] <= 64 and w["l"] >= 0 and w["tol"] == 1e-8, key
    # the headline is the configuration the metric is quoted on (the largest
    # single-GPU one, FP32 against plain FP64); the learned block trains on
    # 200 operators and tests on 20 held-out ones
    assert bench.WORKLOAD["key"] == "chunglu22"
    assert len(bench.WORKLOADS["aniso128"]["train_seeds"]) == 200
    assert bench.HELD_OUT_SEEDS == list(range(2000, 2020))
