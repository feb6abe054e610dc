"""Host-side pieces of bench.py that need no GPU."""
import bench


def line(sm, mx, reasons=("Not Active",) * 4):
    return "0, %d, %d, 500.0, 0x0, %s" % (sm, mx, ", ".join(reasons))


def test_clock_summary_keeps_the_timed_window_only():
    """Samples before the timed window (the idle lead-in) and after it do not
    count; the median comes from the samples under load."""
    stamped = [(0.0, line(2070, 2070)), (0.1, line(1200, 2070)), (0.2, line(1250, 2070)),
               (0.3, line(1300, 2070)), (0.5, line(2070, 2070))]
    c = bench.ClockSampler.summarise(stamped, (0.05, 0.35))
    assert c["sm_mhz"] == 1250 and c["samples"] == 3 and c["samples_in_timed_window"] == 3
    assert c["sm_max_mhz"] == 2070 and c["reasons"] == []


def test_clock_summary_reports_throttle_reasons():
    active = ("Not Active", "Active", "Not Active", "Active")
    stamped = [(1.0, line(1800, 2070, active)), (1.02, line(1810, 2070))]
    c = bench.ClockSampler.summarise(stamped, (0.9, 1.1))
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_short_window_falls_back_to_all_samples():
    """A window shorter than one sampling interval holds no sample: all are
    used, and the count inside is reported as 0."""
    stamped = [(0.0, line(2070, 2070)), (0.02, line(2060, 2070))]
    c = bench.ClockSampler.summarise(stamped, (0.005, 0.006))
    assert c["samples"] == 2 and c["samples_in_timed_window"] == 0
    assert bench.ClockSampler.summarise([], None)["sm_mhz"] is None
