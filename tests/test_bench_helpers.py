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
    # Q1 single-pass CG: x, r, p read and written (24 B per node) and K once per cell
    nn, nc = 1000, 729
    assert bench.cg_bytes(1, nn, nc) == 4.0 * (6 * nn + nc)
    # Q2 fused CG: the apply (x, y, K per cell) plus 24 B per node of CG vectors;
    # 32.5 B per node when a cell holds eight nodes
    assert bench.cg_bytes(2, 8000, 1000) / 8000 == 32.5
    # a graded mesh runs the fused two-pass iteration and reads 16 B of geometry per cell
    assert bench.cg_bytes(1, nn, nc, graded=True) == 4.0 * (2 * nn + nc) + 24.0 * nn + 16.0 * nc
    # FP64 heat apply: x read, y written, three velocity components at each Gauss point
    assert bench.heat_apply_bytes(1, nn, nc) == 16.0 * nn + 24.0 * 8 * nc
    assert bench.heat_apply_bytes(2, 8000, 1000) == 16.0 * 8000 + 24.0 * 27 * 1000
    # operator apply: x read, y written, K once per cell
    assert bench.apply_bytes_per_node(2, False) == 17.0
    assert bench.apply_bytes_per_node(1, True) == 12.0
    assert bench.apply_flops_per_node(2) == 143.0 and bench.apply_flops_per_node(1) == 242.0


def _tree(tmp_path):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_2103_00081_gb300" / "csrc").mkdir(parents=True)
    for f in ("ht_q1.cu", "ht_ops.cu"):
        shutil.copy(os.path.join(bench.ROOT, "paper_2103_00081_gb300", "csrc", f),
                    root / "paper_2103_00081_gb300" / "csrc")
    return root


def test_traffic_record_is_used_only_for_the_source_it_was_taken_on(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    src = root / "paper_2103_00081_gb300" / "csrc" / "ht_q1.cu"
    recs = [{"workload": "city_q1 512x512x96 Q1", "dram_bytes_per_iteration": 7.0e8,
             "source_sha256": hashlib.sha256(src.read_bytes()).hexdigest()},
            {"workload": "other", "dram_bytes_per_iteration": 1.0, "source_sha256": "0"}]
    (root / "profiles" / "cg_iteration_traffic.json").write_text(json.dumps(recs))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.measured_traffic("city_q1 512x512x96 Q1", 1) == 7.0e8
    assert bench.measured_traffic("another workload", 1) is None
    assert bench.measured_traffic("city_q1 512x512x96 Q1", 2) is None      # taken on the Q1 kernel only
    with open(src, "a") as f:
        f.write("\n// changed\n")
    assert bench.measured_traffic("city_q1 512x512x96 Q1", 1) is None


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


def test_cpu_baseline_reports_rate_fit_and_spmv_bandwidth():
    sc_full = bench.workload("plain_q1")
    cb = bench.cpu_baseline(sc_full, "plain_q1")
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0
    assert len(cb["s_per_step_samples"]) == 2 and all(t > 0 for t in cb["s_per_step_samples"])
    assert cb["exponent"] >= 1.0 and cb["host"]["nproc"] >= 1
    assert cb["spmv"]["gbs"] > 0 and cb["spmv"]["rows"] == 17 ** 3
    # the extrapolation follows the fitted law from the larger sample
    n = cb["nodes_samples"]
    assert cb["s_per_step_full_extrapolated"] == pytest.approx(
        cb["s_per_step_samples"][1] * (sc_full.n_nodes / n[1]) ** cb["exponent"])


def test_ates_workload_and_its_oracle_samples():
    """The ATES benchmark workload is the generator's default mesh, and the
    oracle arm times coarser meshes of the same problem (graded in the same
    way, ascending in size)."""
    sc = bench.workload("ates_table1")
    assert (sc.nx, sc.ny, sc.nz, sc.n_nodes) == (266, 266, 90, 6487299)
    samples = bench.oracle_samples("ates_table1", sc)
    assert len(samples) == 2 and samples[0].n_nodes < samples[1].n_nodes < sc.n_nodes
    for s in samples:
        assert s.spacing is not None and s.name == sc.name
        assert s.pile_temps.shape == (1, 9) and s.wells.shape == (1, 7)


def test_oracle_replicas_on_several_cores():
    """The all-core figure of the CPU baseline: spawned single-threaded
    oracle replicas each time one step of the sample."""
    import scenarios as S
    cores, s = bench.oracle_all_cores(S.config5(nx=16, ny=16, nz=3), n_procs=2, timeout_s=120.0)
    assert cores == 2 and 0.0 < s < 60.0
