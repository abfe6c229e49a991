"""Host logic of the benchmark, without a GPU: the clock record taken during
the timed region (median SM clock, the throttle reasons that were active),
the percentile used for per-step latencies, and the reading of the measured
peaks."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.out = "\n".join(lines) + "\n"
    return c


def test_clock_summary_median_and_reasons():
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    c = _sampler([
        "0, 2070, 2070, 700.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ])
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_skips_bad_rows():
    c = _sampler([
        "0, [N/A], 2070, 700, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1500, 2070, 900, 0x40, Not Active, Active, Not Active, Not Active",
        "garbage",
        "0, 1600, 2070, 900, 0x20, Not Active, Not Active, Active, Not Active",
    ])
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == 1550.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = _sampler([]).summary()
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_percentile_nearest_rank():
    xs = list(range(1, 101))                 # 1..100
    assert bench.percentile(xs, 50) == 51    # round(0.5 * 99) = 50 -> 51
    assert bench.percentile(xs, 99) == 99
    assert bench.percentile(xs, 100) == 100
    assert bench.percentile(xs, 0) == 1
    assert bench.percentile([3.0], 99) == 3.0
    assert bench.percentile([], 50) is None
    assert bench.percentile([5, 1, 3], 50) == 3   # unsorted input


def test_load_peaks_flat_nested_missing_and_partial(tmp_path):
    p = tmp_path / "peaks.json"
    p.write_text('{"hbm_gbs": 6789.5, "bf16_tflops": 1907.0, "bf16_tflops_sustained": 1700}')
    pk, src = bench.load_peaks(str(p))
    assert src == "measured" and pk["hbm_gbs"] == 6789.5 and pk["bf16_tflops_sustained"] == 1700
    p.write_text('{"gpu": {"name": "GB300", "peaks": {"hbm_gbs": 7000, "bf16_tflops": 2000}}}')
    pk, src = bench.load_peaks(str(p))
    assert src == "measured" and pk["hbm_gbs"] == 7000.0 and pk["bf16_tflops"] == 2000.0
    p.write_text('{"hbm_gbs": 7000}')
    pk, src = bench.load_peaks(str(p))
    assert pk == {"hbm_gbs": 7000.0, "bf16_tflops": 1900.0} and "fallback: bf16_tflops" in src
    p.write_text("not json")
    assert bench.load_peaks(str(p)) == (bench.FALLBACK_PEAKS, "fallback")
    assert bench.load_peaks(str(tmp_path / "absent.json"))[1] == "fallback"
    p.write_text('{"hbm_gbs": "n/a", "bf16_tflops": true}')
    assert bench.load_peaks(str(p))[1] == "fallback"


def test_section_reports_errors_in_place():
    assert bench.section("ok", lambda: {"a": 1}) == {"a": 1}
    r = bench.section("serving_32_streams", lambda: 1 / 0)
    assert r == {"error": "serving_32_streams: ZeroDivisionError: division by zero"}
