"""bench.py's clock record during the timed region, against a fake
nvidia-smi on PATH (no GPU, no NVML): the median SM clock under load, the
maximum clock and the throttle reasons seen, which decide whether a run is
kept (sw_power_cap) or rejected (hw_slowdown and the thermal reasons)."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

ROWS = [
    "0, 2070, 2070, 900.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 2055, 2070, 1390.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 345, 2070, 110.00, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active",
    "0, 2040, 2070, 1400.00, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
    "[N/A]",
]


def _fake_smi(tmp_path, monkeypatch, rows):
    exe = tmp_path / "nvidia-smi"
    body = "".join(f"echo '{r}'\n" for r in rows)
    exe.write_text("#!/bin/sh\n" + body + "exec sleep 30\n")
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")


def _sample(tmp_path, monkeypatch, rows):
    _fake_smi(tmp_path, monkeypatch, rows)
    c = bench.Clocks(0)
    deadline = time.time() + 10
    while time.time() < deadline and open(c.f.name).read().count("\n") < len(rows):
        time.sleep(0.05)
    return c.stop()


def test_loaded_median_max_and_reasons(tmp_path, monkeypatch):
    rec = _sample(tmp_path, monkeypatch, ROWS)
    # the idle 345 MHz sample is not "under load"; the malformed row is skipped
    assert rec["samples"] == 4
    assert rec["sm_mhz"] == 2055.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clean_run_has_no_reasons(tmp_path, monkeypatch):
    rec = _sample(tmp_path, monkeypatch, ROWS[:1])
    assert rec["reasons"] == [] and rec["sm_mhz"] == 2070.0


def test_missing_tool_is_reported(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))  # no nvidia-smi anywhere
    rec = bench.Clocks(0).stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]
