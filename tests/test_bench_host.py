"""Host-side logic of bench.py: clock records and their rejection rule.

A timed region whose clock samples show a hardware or thermal slowdown, or an
SM clock stuck far below its maximum with no throttle reason (a leftover
clock lock), is taken once more; a power cap alone is kept. The sampler reads
nvidia-smi's CSV from a pipe: here a stand-in process prints fixed lines.
"""
import subprocess
import threading

import bench


def _sampler_with(lines: str) -> bench.ClockSampler:
    cs = bench.ClockSampler(0)
    cs.proc = subprocess.Popen(["printf", lines], stdout=subprocess.PIPE, text=True)
    cs.lines = []
    cs.reader = threading.Thread(target=lambda: cs.lines.extend(cs.proc.stdout), daemon=True)
    cs.reader.start()
    cs.proc.wait(timeout=10)
    return cs


def test_power_cap_is_kept_and_median_under_load():
    cs = _sampler_with("0, 1400, 2032, 900, 0x4, Not Active, Not Active, Not Active, Active\n"
                       "0, 1300, 2032, 950, 0x4, Not Active, Not Active, Not Active, Active\n"
                       "0, 345, 2032, 120, 0x1, Not Active, Not Active, Not Active, Not Active\n")
    clk = cs.stop()
    assert clk["reasons"] == ["sw_power_cap"] and clk["samples"] == 3
    assert clk["sm_mhz"] == 1350.0 and clk["sm_max_mhz"] == 2032.0   # the idle sample is not under load
    assert bench.clocks_rejected(clk) is None


def test_thermal_and_hardware_slowdowns_are_rejected():
    cs = _sampler_with("0, 1100, 2032, 900, 0x48, Active, Not Active, Active, Not Active\n")
    clk = cs.stop()
    assert clk["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.clocks_rejected(clk) == "hw_slowdown+sw_thermal_slowdown"


def test_clock_stuck_low_without_reason_is_rejected():
    assert bench.clocks_rejected({"sm_mhz": 900.0, "sm_max_mhz": 2032.0, "reasons": []}) is not None
    assert bench.clocks_rejected({"sm_mhz": 1900.0, "sm_max_mhz": 2032.0, "reasons": []}) is None


def test_missing_nvidia_smi_is_reported_not_rejected():
    cs = bench.ClockSampler(0)
    cs.proc = None
    clk = cs.stop()
    assert clk["reasons"] == ["nvidia-smi unavailable"] and bench.clocks_rejected(clk) is None
