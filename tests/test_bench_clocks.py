"""bench.py's clock record: only the nvidia-smi samples stamped inside the timed region
count (host logic, no GPU)."""
import datetime

import bench


def _line(t, sm, reasons=()):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    flags = ["Active" if nm in reasons else "Not Active"
             for nm in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")]
    return ", ".join([ts, "0", str(sm), "2070", "950.00", "0x0000000000000000"] + flags)


def test_samples_outside_the_region_are_dropped():
    t0 = 1_700_000_000.0
    out = "\n".join([_line(t0 - 2.0, 1200, ("hw_slowdown",)), _line(t0 + 0.05, 2070), _line(t0 + 0.15, 2055),
                     _line(t0 + 0.25, 2070, ("sw_power_cap",)), _line(t0 + 3.0, 900)])
    c = bench.ClockSampler.summarise(out, t0, t0 + 0.3)
    assert c["samples"] == 3 and c["window"] == "timed region"
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_no_sample_inside_falls_back_to_all():
    t0 = 1_700_000_000.0
    out = "\n".join([_line(t0 - 2.0, 2070), "garbage line", _line(t0 + 5.0, 2000)])
    c = bench.ClockSampler.summarise(out, t0, t0 + 0.1)
    assert c["samples"] == 2 and c["window"].startswith("all samples")


def test_unparsed_stamp_keeps_the_sample():
    t0 = 1_700_000_000.0
    line = _line(t0, 2070).split(", ")
    line[0] = "not a time"
    c = bench.ClockSampler.summarise(", ".join(line), t0, t0 + 0.1)
    assert c["samples"] == 1 and c["sm_mhz"] == 2070.0
