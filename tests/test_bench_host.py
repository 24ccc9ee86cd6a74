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


def test_roofline_from_profiled_kernel_times():
    """The dominant kernel's roofline from per-kernel totals over K profiled
    steps (the figures of a measured 1M-point run)."""
    launches = 3787
    prof = {"k_cavity_w<3>": {"ms": 319.261, "launches": launches, "bytes": 36927271.45814629 * launches,
                              "flops": 487.258486271189e9 * 0.319261},
            "k_insert_w<3>": {"ms": 103.117, "launches": launches, "bytes": 0.0, "flops": 0.0}}
    r = bench.make_roofline(prof, [150.0] * 5, 1_000_000, 5, {"hbm_gbs": 6800.7}, "measured")
    assert r["kernel"] == "k_cavity_w<3>" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(438.02, rel=1e-4)
    assert r["frac"] == pytest.approx(438.02 / 6800.7, rel=1e-4)
    assert r["share_of_step"] == pytest.approx(319.261 / 750.0)
    assert r["alu"]["achieved"] == pytest.approx(0.48726, rel=1e-4)
    assert r["alu"]["frac"] == pytest.approx(0.48726 / bench.FP32_PEAK_TFLOPS, rel=1e-4)
    stored = bench.stored_cavity_traffic()
    if stored is not None:   # DRAM bytes per point scaled to one launch (launches per step = 3787 / 5)
        assert r["traffic"] == pytest.approx(stored * 1_000_000 / (launches / 5))
    assert bench.make_roofline({}, [], 1, 1, {"hbm_gbs": 1.0}, "fallback") is None
