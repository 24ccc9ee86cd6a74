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


def test_roofline_from_profiled_kernel_times():
    """The dominant kernel's roofline from per-kernel totals over 5 profiled
    steps: 320 B and 2.3 kflop per triangulated point (1,265,715 points per
    step: n + eta + |vertices(B)| of a measured 1M-point run) over the
    kernel's time per step (319.261 ms / 5 = 63.8522 ms)."""
    launches = 3787
    prof = {"k_cavity_w<3>": {"ms": 319.261, "launches": launches, "bytes": 36927271.45814629 * launches,
                              "flops": 220.0 * 141e6 * 5},
            "k_insert_w<3>": {"ms": 103.117, "launches": launches, "bytes": 0.0, "flops": 0.0}}
    fma = {"fp64": 1.2, "fp32": 70.0}
    r = bench.make_roofline(prof, [150.0] * 5, 1_265_715, 3, 5, {"hbm_gbs": 6800.7}, "measured", fma,
                            n=1_000_000)
    assert r["kernel"] == "k_cavity_w<3>" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    # 320 x 1,265,715 = 405,028,800 B per step over 63.8522 ms
    assert r["achieved"] == pytest.approx(6.34322, rel=1e-4)
    assert r["frac"] == pytest.approx(6.34322 / 6800.7, rel=1e-4)
    assert r["bytes_per_launch"] == pytest.approx(405_028_800 / (3787 / 5), rel=1e-9)
    assert r["gather_bytes_per_launch"] == pytest.approx(36927271.45814629)
    assert r["share_of_step"] == pytest.approx(319.261 / 750.0)
    # 2,300 x 1,265,715 = 2.9111445e9 flops per step over 63.8522 ms
    assert r["fp64"]["achieved"] == pytest.approx(0.0455919, rel=1e-4)
    assert r["fp64"]["frac"] == pytest.approx(0.0455919 / 1.2, rel=1e-4)
    assert r["fp32"]["frac"] == pytest.approx(0.0455919 / 70.0, rel=1e-4)
    assert r["conflict_tests_per_point"] == pytest.approx(141e6 / 1_265_715)
    stored = bench.stored_cavity_traffic()
    if stored is not None:   # DRAM bytes per input point scaled to one launch (launches per step = 3787 / 5)
        assert r["traffic"] == pytest.approx(stored * 1_000_000 / (launches / 5))
    assert bench.make_roofline({}, [], 1, 3, 1, {"hbm_gbs": 1.0}, "fallback") is None


def test_sample_size_flags():
    """--frac: a fraction, 'sqrt' (the library's 0) or 'logn' (rounds up to ceil(log2 n))."""
    import math
    assert bench.parse_frac(None, 0.005, 10) == 0.005
    assert bench.parse_frac("0.02", 0.005, 10) == 0.02
    assert bench.parse_frac("sqrt", 0.005, 10) == 0.0
    for n in (1_000_000, 4_000_000, 10_000):
        f = bench.parse_frac("logn", 0.005, n)
        assert math.ceil(f * n) == math.ceil(math.log2(n))
