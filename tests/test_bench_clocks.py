"""The bench's clock sampler against a fake nvidia-smi on PATH (no GPU): it waits for the first
sample, takes the median SM clock under load and reports every throttle reason that was active
in any sample, since a run that saw a thermal or hardware slowdown is not a valid measurement."""
import os
import stat
import time

import pytest

import bench

# index, clocks.sm, clocks.max.sm, power.draw, active mask, hw_slowdown, hw_thermal_slowdown,
# sw_thermal_slowdown, sw_power_cap
ROWS = [
    "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2070, 2070, 1100.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 2070, 2070, 1000.0, 0x0000000000000000, Not Active, Active, Not Active, Not Active",
    "garbage line",
]


def fake_smi(tmp_path, rows, delay_s=0.3):
    script = tmp_path / "nvidia-smi"
    body = "\n".join(f"echo '{r}'; sleep 0.05" for r in rows)
    script.write_text(f"#!/bin/sh\nsleep {delay_s}\n{body}\nexec sleep 5\n")
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_clock_sampler_waits_and_parses(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", fake_smi(tmp_path, ROWS) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler("0")
    assert s.p is not None
    t0 = time.perf_counter()
    s.wait_first()
    assert time.perf_counter() - t0 >= 0.25          # returned only once a sample was written
    time.sleep(0.5)
    c = s.stop()
    assert c["samples"] == 4                          # the malformed line is skipped
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler("0")
    s.wait_first(timeout_s=0.2)
    c = s.stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]


@pytest.mark.parametrize("delay_s", [3.0])
def test_clock_sampler_wait_is_bounded(tmp_path, monkeypatch, delay_s):
    monkeypatch.setenv("PATH", fake_smi(tmp_path, ROWS[:1], delay_s) + os.pathsep +
                       os.environ["PATH"])
    s = bench.ClockSampler("0")
    t0 = time.perf_counter()
    s.wait_first(timeout_s=0.5)
    assert time.perf_counter() - t0 < 2.0
    c = s.stop()
    assert c["samples"] == 0 and c["sm_mhz"] is None
