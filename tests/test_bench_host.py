"""Host logic of bench.py that needs no GPU: the clock-sample parser that decides which throttle
reasons a measured line reports, and the roofline peak source."""
import bench


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.lines = lines
    return c.summary()


def test_clock_summary_reports_medians_and_active_reasons():
    ok = "0, 2032, 2032, 710.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    slow = "0, 1700, 2032, 1080.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active"
    cap = "0, 1900, 2032, 1099.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    s = _sampler([ok, ok, slow, cap, "garbage", "0, [N/A], 2032, 1.0, 0x0, a, b, c, d"])
    assert s["samples"] == 4
    assert s["sm_mhz"] == 1966.0                      # median of 2032, 2032, 1700, 1900
    assert s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples_says_so():
    s = _sampler([])
    assert s["samples"] == 0 and s["reasons"] == ["unsampled"]


def test_clean_run_has_no_reasons():
    ok = "0, 2032, 2032, 500.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    assert _sampler([ok] * 3)["reasons"] == []


def test_thermal_reasons_are_named():
    th = "0, 1500, 2032, 900.0, 0x0000000000000060, Not Active, Active, Active, Not Active"
    assert _sampler([th])["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_peaks_come_from_the_measured_file_when_present():
    pk, src = bench.peaks()
    assert src in ("measured", "fallback")
    assert pk["bf16_tflops"] > 0 and pk.get("sm_max_mhz", 2032.0) > 0
