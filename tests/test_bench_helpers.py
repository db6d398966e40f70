"""CPU checks of the measurement helpers in bench.py: the algorithmic bytes per
node, the traffic record's source check, the peak fallback and the clock
record parser."""
import hashlib
import json
import os
import shutil

import pytest

import bench


def test_algorithmic_bytes_per_node():
    # fused CG iteration: 10 FP32 vector words per node plus K once per cell
    assert bench.fused_cg_bytes_per_node(2, True) == 40.5      # Q2: a cell per 8 nodes
    assert bench.fused_cg_bytes_per_node(1, True) == 44.0      # Q1: a cell per node
    # operator apply: x read, y written, K once per cell
    assert bench.apply_bytes_per_node(2, False) == 17.0
    assert bench.apply_bytes_per_node(1, True) == 12.0
    assert bench.apply_flops_per_node(2) == 143.0 and bench.apply_flops_per_node(1) == 242.0


def _tree(tmp_path):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_2103_00081_gb300" / "csrc").mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "fused_cg_traffic.json"), root / "profiles")
    shutil.copy(os.path.join(bench.ROOT, "paper_2103_00081_gb300", "csrc", "ht_ops.cu"),
                root / "paper_2103_00081_gb300" / "csrc")
    return root


def test_traffic_record_is_used_only_for_the_source_it_was_taken_on(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    rec = json.load(open(root / "profiles" / "fused_cg_traffic.json"))
    # a record taken on the copied source
    with open(root / "paper_2103_00081_gb300" / "csrc" / "ht_ops.cu", "rb") as f:
        rec["source_sha256"] = hashlib.sha256(f.read()).hexdigest()
    with open(root / "profiles" / "fused_cg_traffic.json", "w") as f:
        json.dump(rec, f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.measured_traffic(rec["workload"]) == rec["dram_bytes_per_iteration"]
    assert bench.measured_traffic("another workload") is None
    with open(root / "paper_2103_00081_gb300" / "csrc" / "ht_ops.cu", "a") as f:
        f.write("\n// changed\n")
    assert bench.measured_traffic(rec["workload"]) is None


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pk = bench.peaks()
    assert pk["source"] == "fallback" and pk["hbm_gbs"] == 6800.0
    assert pk["fp32_tflops"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6682.2, "sm_max_mhz": 2070.0}))
    pk = bench.peaks()
    assert pk["source"] == "measured" and pk["hbm_gbs"] == 6682.2


def test_clock_record_parser(tmp_path):
    c = bench.Clocks()
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active\n")
        f.write("1980, 2070, 1390.0, Not Active, Not Active, Not Active, Active\n")
        f.write("2010, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("garbage line\n")
    s = c.summary()
    assert s["sm_mhz"] == 2010 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.path = str(tmp_path / "missing.csv")
    assert c.summary()["reasons"] == ["unsampled"]


def test_cpu_baseline_reports_rate_step_time_and_spmv_bandwidth():
    import types
    args = types.SimpleNamespace(cpu_sample_cells=6)
    sc_full = bench.workload("ates_q2")
    cb = bench.cpu_baseline(args, sc_full)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0
    assert cb["s_per_step_sample"] > 0 and cb["spmv"]["gbs"] > 0
    assert cb["spmv"]["rows"] == (2 * 6 + 1) ** 2 * (2 * 2 + 1)
