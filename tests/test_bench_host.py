"""Host-side helpers of bench.py on the CPU: the clock record taken during
the timed region (median and maximum SM clock, throttle reasons that reject a
run) and the committed traffic figure, read only for the kernel source it was
measured on."""

import bench


def test_clock_summary_median_max_and_reasons():
    ok = "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1395.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    thermal = "0, 1500, 2070, 1100.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active"
    s = bench.summarize_clocks([ok, ok, capped])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s = bench.summarize_clocks([ok, thermal, "garbage", "", "0, [N/A], 2070, 1, 0, a, b, c, d"])
    assert s["samples"] == 2 and s["sm_mhz"] == (2070.0 + 1500.0) / 2
    assert s["reasons"] == ["hw_thermal_slowdown"]
    assert bench.summarize_clocks([]) is None
    assert bench.summarize_clocks(["garbage"]) is None


def test_traffic_is_reported_only_for_the_profiled_kernel_source(monkeypatch):
    t = bench._traffic("gs_vol_f64")
    with open(bench.os.path.join(bench.ROOT, "profiles", "traffic_gs_fp64_config2.md")) as fh:
        text = fh.read()
    recorded = [ln.split(":", 1)[1].strip() for ln in text.splitlines() if ln.startswith("kernel_hash:")]
    assert len(recorded) == 1
    if recorded[0] == bench._kernel_hash():
        assert t is not None and t > 0
    else:
        assert t is None
    monkeypatch.setattr(bench, "_kernel_hash", lambda: "0" * 16)
    assert bench._traffic("gs_vol_f64") is None
