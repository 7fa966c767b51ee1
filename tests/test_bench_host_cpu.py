"""Host logic of bench.py without a GPU: the ping-pong schedule over the scan
sequence and the clock sampler's parsing of nvidia-smi output (a fake
nvidia-smi on PATH prints the rows)."""
import os
import stat
import sys

ROOT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..")
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_ping_pong_schedule():
    s = bench.ping_pong(12, 4)
    assert s == [0, 1, 2, 3, 2, 1, 0, 1, 2, 3, 2, 1]
    s = bench.ping_pong(500, 100)
    assert all(abs(a - b) == 1 for a, b in zip(s, s[1:]))   # neighbouring scans: small window moves
    assert min(s) == 0 and max(s) == 99


def test_clock_sampler_parses_rows(tmp_path, monkeypatch):
    rows = [
        "2026/01/01 00:00:00.000, 0, 1000, 2070, 300.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/01/01 00:00:00.100, 0, 2070, 2070, 1200.5, 0x4, Not Active, Not Active, Not Active, Active",
        "2026/01/01 00:00:00.200, 0, 2070, 2070, 1250.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/01/01 00:00:00.300, 0, 2055, 2070, 1190.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "a malformed line",
    ]
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n" + "".join(f"echo '{r}'\n" for r in rows) + "exec sleep 30\n")
    fake.chmod(fake.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    c = bench.ClockSampler(None)
    c.mark_start()
    c.mark_end()
    out = c.stop()
    assert out["samples"] == 4
    assert out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2070.0            # median of the loaded (upper) half
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    out = bench.ClockSampler(None).stop()
    assert out["samples"] == 0 and out["sm_mhz"] is None
