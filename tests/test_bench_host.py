"""Host-side pieces of bench.py that need no GPU: a DRAM-traffic record is
reported only while it was taken on the current sigma kernel source."""
import os

import bench


def test_traffic_record_rejected_for_other_source(tmp_path, monkeypatch):
    rec = tmp_path / "profiles"
    rec.mkdir()
    (rec / "traffic_h2o29.txt").write_text("source_sha = 0000000000000000\n"
                                     "alpha_beta.bytes_per_launch = 1e8\n")
    (tmp_path / "paper_2601_16169_gb300").symlink_to(
        os.path.join(bench.ROOT, "paper_2601_16169_gb300"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("alpha_beta") is None
    (rec / "traffic_h2o29.txt").write_text("source_sha = %s\nalpha_beta.bytes_per_launch = 1e8\n"
                                     % bench.kernel_source_hash())
    assert bench.recorded_traffic("alpha_beta") == 1e8
    assert bench.recorded_traffic("same_spin_beta") is None
    assert bench.recorded_traffic("alpha_beta", "scale36") is None  # no record for it


def test_fp64_peak_is_the_derived_one():
    # 152 SMs x 2070 MHz x 4 FP64 flop per clock per SM
    assert abs(bench.FP64_PEAK_TFLOPS - 1.25856) < 1e-9


def test_clock_parsing_reports_throttle_reasons():
    text = ("0, 2070, 2070, 800.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
            "0, 2060, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active\n"
            "0, 2070, 2070, 910.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    c = bench.parse_clocks(text)
    assert c["sm_mhz"] == 2070 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]


def test_default_line_is_the_largest_workload():
    a = bench._args([])
    assert a.workload == "scale36" and a.mode == "headline" and a.gpus == 1
    assert a.warmup >= 3


def test_class_record_fractions():
    prof = {"davidson": dict(regions=2, ms=10.0, flops=1.0e10, bytes=3.3e10)}
    r = bench.class_record(prof, ["davidson"])["davidson"]
    assert abs(r["tflops"] - 1.0) < 1e-12
    assert abs(r["frac_fp64_peak"] - 1.0 / bench.FP64_PEAK_TFLOPS) < 1e-12
    assert abs(r["gbs"] - 3300.0) < 1e-9


def test_oracle_solve_baseline_full8():
    # the whole-solve CPU baseline of the full8 sub-record reaches the stored
    # lowest eigenvalue of the dense full8 Hamiltonian
    from tests.golden import make_golden as mg
    r = bench.oracle_solve("full8")
    assert r["converged"] and r["kind"] == "oracle" and r["seconds"] > 0
    assert abs(r["energies"][0] - mg.read_full8()[0]) <= 1e-9
    assert "full8" in bench.SUBRECORDS
