"""Host-side logic of bench.py and of the ncu-summary script: the roofline traffic read from the ncu summary
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


def test_traffic_script_maps_kernels_to_profiler_families():
    """The ncu kernel names, demangled with or without the template-argument
    casts, go to the library profiler's families; setup kernels go nowhere."""
    from paper_1711_10128_gb300 import traffic as T
    cases = {
        "void trplk::ts_kernel<float, (int)1, (int)32>(trplk::TSArgs<T1>)": "ts_inner",
        "void ts_kernel<double, 3, 64>(TSArgs<T1>)": "ts_update_norm_f64",
        "void ts_kernel<float, 0, 48>(TSArgs<T1>)": "ts_project",
        "void trplk::ts_kernel<double, (int)5, (int)64>(trplk::TSArgs<T1>)": "ts_rotate_f64",
        "void sell_spmv_kernel<float, (bool)1, (bool)1>(long, long, const long *)": "spmv_scaled",
        "void sell_spmv_kernel<double, 0, 1>(long)": "spmv_f64",
        "void dia_spmv_kernel<float, true>(long)": "spmv_scaled",
        "void spmv_kernel<double, false>(long)": "spmv_f64",
        "rotate_tc_kernel(CUtensorMap_st, trplk::RotArgs)": "ts_rotate",
        "void trplk::rr_kernel(int, const double *, int, double *, double *, int *, int)": "rayleigh_ritz",
        "void trplk::validate_csr_kernel(long, long)": None,
    }
    for name, fam in cases.items():
        assert T.family_of(name) == fam, name


def test_traffic_script_reads_raw_and_details_pages(tmp_path):
    """Both ncu CSV layouts give the same launches, in bytes and nanoseconds."""
    from paper_1711_10128_gb300 import traffic as T
    raw = tmp_path / "raw.csv"
    raw.write_text(
        '"ID","Kernel Name","gpu__time_duration.sum","dram__bytes_read.sum","dram__bytes_write.sum"\n'
        '"","","usecond","Mbyte","Kbyte"\n'
        '"0","void ts_kernel<float, 1, 32>(TSArgs<T1>)","2.5","1.5","4"\n'
        '"1","void trplk::validate_csr_kernel(long)","1,000","n/a","0"\n')
    details = tmp_path / "details.csv"
    rows = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    for i, (name, vals) in enumerate([("void ts_kernel<float, 1, 32>(TSArgs<T1>)", ("2.5", "1.5", "4")),
                                      ("void trplk::validate_csr_kernel(long)", ("1,000", "n/a", "0"))]):
        for metric, unit, v in zip(T.METRICS, ("usecond", "Mbyte", "Kbyte"), vals):
            rows.append(f'"{i}","{name}","{metric}","{unit}","{v}"')
    details.write_text("\n".join(rows) + "\n")
    for path in (raw, details):
        got = T.read_launches(str(path))
        assert len(got) == 2
        name, fam, t, rd, wr = got[0]
        assert fam == "ts_inner" and abs(t - 2500.0) < 1e-9 and abs(rd - 1.5e6) < 1e-6 and abs(wr - 4e3) < 1e-9
        assert got[1][1] is None and abs(got[1][2] - 1e6) < 1e-6 and got[1][3] is None and got[1][4] == 0.0


def test_traffic_script_records_ratios_only_where_launch_counts_agree(tmp_path, monkeypatch):
    from paper_1711_10128_gb300 import traffic as T
    raw = tmp_path / "raw.csv"
    lines = ['"ID","Kernel Name","gpu__time_duration.sum","dram__bytes_read.sum","dram__bytes_write.sum"',
             '"","","nsecond","byte","byte"']
    for i in range(3):   # three first-pass launches, 900 + 100 DRAM bytes each
        lines.append(f'"{i}","void ts_kernel<float, 1, 32>(TSArgs<T1>)","300","900","100"')
    lines.append('"3","void sell_spmv_kernel<float, 1, 1>(long)","600","2000","0"')
    raw.write_text("\n".join(lines) + "\n")
    prof = tmp_path / "prof.json"
    prof.write_text("some log line\n" + json.dumps({"workload": "w", "solves": 1, "families": {
        "ts_inner": {"launches": 3, "algorithmic_bytes": 2500.0},
        "spmv_scaled": {"launches": 2, "algorithmic_bytes": 4000.0},   # count differs: not recorded
        "rayleigh_ritz": {"launches": 1, "algorithmic_bytes": 0.0}}}) + "\n")
    out = tmp_path / "traffic.json"
    md = tmp_path / "launches.md"
    monkeypatch.setattr(T, "OUT", str(out))
    monkeypatch.setattr(sys, "argv", ["traffic", str(raw), str(prof), "--command", "ncu ...",
                                      "--launches-md", str(md)])
    T.main()
    data = json.load(open(out))
    assert set(data) == {"w/ts_inner"}
    e = data["w/ts_inner"]
    assert abs(e["dram_per_algorithmic_byte"] - 3000.0 / 2500.0) < 1e-12 and e["launches"] == 3
    assert e["sha256"] == T.sources_sha(e["sources"]) and e["sources"]
    text = md.read_text()
    assert "| `ts_kernel<float, 1, 32>` | ts_inner | 3 | 0.9 | 0.6000 |" in text
    assert "| `sell_spmv_kernel<float, 1, 1>` | spmv_scaled | 1 | 0.6 | 0.4000 |" in text
