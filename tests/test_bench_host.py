"""Host logic of the benchmark that needs no GPU: the summary of the
nvidia-smi clock samples taken during the timed region (median SM clock,
maximum clock, throttle reasons seen active)."""


def test_clock_summary_of_nvidia_smi_rows():
    import bench
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1950, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1, 900, 2070, 300.0, 0x40, Active, Not Active, Not Active, Not Active",  # another GPU
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",  # unreadable clock
        "garbage",
    ]
    out = bench.ClockSampler.summarise(rows, [0])
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    both = bench.ClockSampler.summarise(rows, None)
    assert both["samples"] == 4 and both["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler.summarise(["garbage"], None) is None
