"""Host logic of bench.py, on the CPU: the DRAM-traffic lookup keyed by the library's
source hash, the peak denominators and their fallback, and the clock-record summary
(the throttle reasons that reject a run)."""
import json

import pytest

import bench


def write_traffic(path, sha, workload="3d_f32_512 NOA 0.001", kernels=None):
    kernels = {"tile_pass": {"dram_bytes_read": 100, "dram_bytes_write": 23}} if kernels is None else kernels
    path.write_text(json.dumps({"workload": workload, "source_sha256": sha, "kernels": kernels}))


def test_traffic_is_reported_only_for_the_sources_it_was_captured_with(tmp_path, monkeypatch):
    p = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(p))
    sha = bench.library_source_sha256()
    write_traffic(p, sha)
    assert bench.measured_traffic("tile_pass", "3d_f32_512 NOA 0.001") == 123
    assert bench.measured_traffic("decode", "3d_f32_512 NOA 0.001") is None      # not captured
    assert bench.measured_traffic("tile_pass", "3d_f32_256 NOA 0.001") is None   # another workload
    write_traffic(p, "0" * 64)                                                  # stale counters
    assert bench.measured_traffic("tile_pass", "3d_f32_512 NOA 0.001") is None
    p.write_text("{not json")
    assert bench.measured_traffic("tile_pass", "3d_f32_512 NOA 0.001") is None
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(tmp_path / "missing.json"))
    assert bench.measured_traffic("tile_pass", "3d_f32_512 NOA 0.001") is None


def test_source_hash_follows_every_library_source(tmp_path, monkeypatch):
    from paper_2603_26968_b300 import build
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cuh"
    a.write_text("x")
    b.write_text("y")
    monkeypatch.setattr(build, "sources", lambda: [a, b])
    h1 = bench.library_source_sha256()
    b.write_text("y // a comment")
    assert bench.library_source_sha256() != h1
    b.write_text("y")
    assert bench.library_source_sha256() == h1


def test_peaks_read_the_measured_file_or_fall_back(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6400.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6451.8, "bf16_tflops": 1800}))
    assert bench.peaks() == (6451.8, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"bf16_tflops": 1800}))
    assert bench.peaks() == (6400.0, "fallback")


def clock_line(sm, smax, active="Not Active", hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {smax}, 700.5, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_median_max_and_reasons():
    s = bench.ClockSampler(0)
    s.lines = [clock_line(2032, 2032), clock_line(1980, 2032, cap="Active"), clock_line(2032, 2032),
               "garbage", "0, [N/A], 2032, 1, 0, a, b, c, d"]
    out = s.summary()
    assert out["sm_mhz"] == 2032.0 and out["sm_max_mhz"] == 2032.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    s.lines = [clock_line(1200, 2032, hwt="Active"), clock_line(1100, 2032, hw="Active")]
    out = s.summary()
    assert out["sm_mhz"] == pytest.approx(1150.0)
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0)
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}


def test_host_cpu_record():
    hc = bench.host_cpu()
    assert hc["nproc"] >= 1 and isinstance(hc["cpu_model"], str) and hc["cpu_model"]
