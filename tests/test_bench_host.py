"""Host-side pieces of bench.py that need no GPU: a DRAM-traffic record is
reported only while it was taken on the current sigma kernel source."""
import os

import bench


def test_traffic_record_rejected_for_other_source(tmp_path, monkeypatch):
    rec = tmp_path / "profiles"
    rec.mkdir()
    (rec / "traffic.txt").write_text("source_sha = 0000000000000000\n"
                                     "alpha_beta.bytes_per_launch = 1e8\n")
    (tmp_path / "paper_2601_16169_gb300").symlink_to(
        os.path.join(bench.ROOT, "paper_2601_16169_gb300"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("alpha_beta") is None
    (rec / "traffic.txt").write_text("source_sha = %s\nalpha_beta.bytes_per_launch = 1e8\n"
                                     % bench.kernel_source_hash())
    assert bench.recorded_traffic("alpha_beta") == 1e8
    assert bench.recorded_traffic("same_spin_beta") is None


def test_fp64_peak_is_the_derived_one():
    # 152 SMs x 2070 MHz x 4 FP64 flop per clock per SM
    assert abs(bench.FP64_PEAK_TFLOPS - 1.25856) < 1e-9
