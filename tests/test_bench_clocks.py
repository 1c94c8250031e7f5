"""The bench's clock record (host logic, no GPU): nvidia-smi samples taken
during the timed region are reduced to the median SM clock, the maximum
clock and the throttle reasons seen active; a fake nvidia-smi on PATH stands
in for the real one."""
import os
import stat
import time

import bench


def row(sm, mx, *active):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in active else "Not Active" for n in names]
    return ["0", str(sm), str(mx), "900.5", "0x0000000000000000", *flags]


def test_summarize_median_max_and_reasons():
    rows = [row(2070, 2070), row(1980, 2070, "sw_power_cap"), row(2070, 2070), ["garbage"]]
    out = bench.ClockSampler.summarize(rows)
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_summarize_flags_every_throttle_kind():
    rows = [row(1400, 2070, "hw_slowdown"), row(1400, 2070, "hw_thermal_slowdown", "sw_thermal_slowdown")]
    out = bench.ClockSampler.summarize(rows)
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1400.0


def test_summarize_without_samples():
    assert bench.ClockSampler.summarize([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                                                "samples": 0}


def test_sampler_reads_a_fake_nvidia_smi(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 2070, 2070, 1200.00, 0x0, Not Active, Not Active, Not Active, Active'\n"
                    "echo '0, 2055, 2070, 1210.00, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    s = bench.ClockSampler(0)
    for _ in range(50):
        if len(s.rows) >= 2:
            break
        time.sleep(0.1)
    out = s.stop()
    assert out["samples"] == 2 and out["sm_max_mhz"] == 2070.0 and out["reasons"] == ["sw_power_cap"]
    assert out["sm_mhz"] == (2070.0 + 2055.0) / 2
