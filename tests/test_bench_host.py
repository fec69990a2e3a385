"""bench.py's host helpers on CPU: the clock sampler's summary of
nvidia-smi lines (median SM clock, maximum, throttle reasons seen) and the
roofline record (fraction of the FP64 peak, DRAM bandwidth from a traffic
figure)."""
import bench


def test_clock_summary_reports_median_and_reasons():
    cs = bench.ClockSampler(0)
    with open(cs.out.name, "w") as f:
        f.write("0, 2070, 2070, 950.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2070, 2070, 1001.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("garbage line\n")
        f.write("0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_hw_slowdown():
    cs = bench.ClockSampler(0)
    with open(cs.out.name, "w") as f:
        f.write("0, 1500, 2070, 700.0, 0x8, Active, Not Active, Active, Not Active\n")
    s = cs.summary()
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and s["sm_mhz"] == 1500.0


def test_roofline_record(monkeypatch):
    monkeypatch.setattr(bench, "measured_hbm_gbs", lambda: 6785.9)
    r = bench.roofline(0.25, 10.0e9, 20.0)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["frac"] - 0.25 / bench.FP64_PEAK_TFLOPS) < 1e-12
    assert abs(r["dram_gbs"] - 500.0) < 1e-9                 # 10 GB in 20 ms
    assert abs(r["dram_frac_of_measured_hbm"] - 500.0 / 6785.9) < 1e-12
    r = bench.roofline(0.25, None, 20.0)
    assert r["traffic"] is None and "dram_gbs" not in r
    r = bench.roofline(0.25, (10.0e9, "captured with another schedule"), 20.0)
    assert r["traffic"] == 10.0e9 and r["traffic_schedule"] == "captured with another schedule"
