"""Host-side pieces of bench.py (no GPU): the clock record, the peak and
DRAM-traffic lookups, the derived FP32 roof."""
import json

import pytest

import bench


def test_clock_record_median_max_and_reasons():
    c = bench.ClockSampler(0)
    c.rows = [["0", "2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "1980", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["0", "2010", "2070", "1200.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["garbage"]]
    r = c.stop()
    assert r["sm_mhz"] == 2010.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 4


def test_peaks_measured_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench.load_peaks()
    assert src == "fallback" and peaks["hbm_gbs"] == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5}))
    peaks, src = bench.load_peaks()
    assert src == "measured" and peaks["hbm_gbs"] == 7000.5


def test_stored_traffic_only_for_the_kernel_it_was_taken_on(monkeypatch):
    fp = bench.cavity_fingerprint()
    assert len(fp) == 40
    stored = bench.stored_cavity_traffic()
    if stored is None:
        pytest.skip("the committed capture predates the current kernel source")
    assert stored > 0
    monkeypatch.setattr(bench, "cavity_fingerprint", lambda: "0" * 40)
    assert bench.stored_cavity_traffic() is None


def test_derived_fp32_roof():
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2 * 2.07e-3)
