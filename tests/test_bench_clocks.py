"""bench.py's clock record from nvidia-smi samples (the JSON line's "clocks"):
the median SM clock under load, the largest maximum clock, and every throttle
reason that was active in any sample -- the fields a run is accepted or
rejected by. The samples are the CSV rows of the query, as nvidia-smi prints
them (no header, no units)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_clk", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _row(sm, mx, power, active, hw="Not Active", hwt="Not Active", swt="Not Active",
         cap="Not Active"):
    return [v.strip() for v in f"{sm}, {mx}, {power}, {active}, {hw}, {hwt}, {swt}, {cap}".split(",")]


def test_clean_run():
    b = _bench()
    c = b.ClockSampler()
    c.samples = [_row(2070, 2070, 900.5, "0x0000000000000000") for _ in range(5)]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}


def test_median_and_reasons():
    b = _bench()
    c = b.ClockSampler()
    c.samples = [_row(2070, 2070, 1200, "0x4", cap="Active"),
                 _row(1965, 2070, 1390, "0x4", cap="Active"),
                 _row(1980, 2070, 1380, "0x40", hwt="Active"),
                 _row(2070, 2070, 1000, "0x0")]
    s = c.summary()
    assert s["sm_mhz"] == 2025.0  # median of four
    assert s["sm_max_mhz"] == 2070.0
    # power cap kept and noted; a thermal slowdown is listed (the run is rejected)
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_every_rejecting_reason_is_seen():
    b = _bench()
    c = b.ClockSampler()
    c.samples = [_row(2070, 2070, 500, "0x8", hw="Active"),
                 _row(2070, 2070, 500, "0x20", swt="Active")]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_unparsable_and_missing_samples():
    b = _bench()
    c = b.ClockSampler()
    assert c.summary()["reasons"] == ["unsampled"]  # no sample at all
    c.samples = [["[N/A]", "[N/A]", "[N/A]", "[N/A]"], _row(1500, 2070, 300, "0x0")]
    s = c.summary()
    assert s["sm_mhz"] == 1500.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == []
