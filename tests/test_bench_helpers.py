"""Host-side helpers of bench.py that need no GPU: the summary of the clock
record taken during the timed region."""
import bench


def test_clock_summary_median_and_reasons():
    lines = [
        "0, 2070, 2070, 812.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 900.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = bench.summarise_clocks(lines)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_empty():
    s = bench.summarise_clocks(["0, 1500, 2070, 1400, 0x48, Active, Active, Not Active, Not Active"])
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    e = bench.summarise_clocks([])
    assert e["sm_mhz"] is None and e["samples"] == 0
