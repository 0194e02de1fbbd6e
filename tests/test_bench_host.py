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


def test_integer_stage_rooflines():
    # one call: 1,000 bytes in 10 records, 400 tokens, 20 recognizer / 30 NER / 40 final spans,
    # 1,100 output bytes; two profiled calls, each stage timed over both
    st = {"n_bytes": 1000, "n_tokens": 400, "n_records": 10, "n_regex_spans": 20, "n_ner_spans": 30,
          "n_final_spans": 40, "n_out_bytes": 1100}
    prof = {"stage_calls": 2, "stage_ms": {"text": 2e-3, "spans": 1e-3, "hash_map": 4e-3, "substitution": 1e-3}}
    out = bench.integer_stages(prof, st, 6000.0, "measured", total_ms=10.0)
    text = 1000 + 12 * 400 + 8 * 11 + 9 * 20          # text once, token table, record offsets, spans
    spans = 400 + 16 * 30 + 9 * 20 + 9 * 40          # labels, NER boundaries, recognizer spans, final spans
    subst = 1000 + 1100 + 49 * 40 + 16 * 11           # text in, output out, final spans, offsets in and out
    assert out["calls"] == 2
    assert out["text"]["alg_bytes"] == text and out["spans"]["alg_bytes"] == spans
    assert out["substitution"]["alg_bytes"] == subst
    # per call: 1e-3 ms for the text stage -> bytes / 1 us
    assert abs(out["text"]["gb_s"] - text / 1e-6 / 1e9) < 1e-9
    assert abs(out["text"]["frac"] - out["text"]["gb_s"] / 6000.0) < 1e-12
    assert abs(out["hash_map"]["spans_per_s"] - 40 / 2e-6) < 1e-3
    assert abs(out["substitution"]["share_of_step"] - 1e-3 / 10.0) < 1e-12
    # no profiled call: no rates, no division by zero
    empty = bench.integer_stages({"stage_calls": 0, "stage_ms": {}}, st, 6000.0, "measured", total_ms=10.0)
    assert empty["text"]["gb_s"] is None and empty["hash_map"]["spans_per_s"] is None
