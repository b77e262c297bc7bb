"""The benchmark's clock record on CPU: `ClockSampler` runs nvidia-smi in
looping mode during the timed region and reports the median SM clock, the
maximum clock and every throttle reason seen active.  A fake nvidia-smi on
PATH stands in for the real one (no GPU here)."""

import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = r"""#!/bin/sh
# fake nvidia-smi: one CSV line every 50 ms until terminated
i=0
while true; do
  case $((i % 3)) in
    0) echo "0, 2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active" ;;
    1) echo "0, 2055, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active" ;;
    2) echo "0, 2070, 2070, 1290.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active" ;;
  esac
  i=$((i + 1))
  sleep 0.05
done
"""


def _fake_path(tmp_path, body):
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    f.write_text(body)
    f.chmod(f.stat().st_mode | stat.S_IXUSR)
    return str(d) + os.pathsep + os.environ.get("PATH", "")


def test_clock_sampler_median_max_and_reasons(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_path(tmp_path, FAKE))
    sys.path.insert(0, ROOT)
    import bench

    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.6)
    rec = s.stop()
    assert rec["samples"] >= 3
    assert rec["sm_mhz"] in (2055.0, 2070.0)
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    empty = tmp_path / "empty"
    empty.mkdir()
    monkeypatch.setenv("PATH", str(empty))
    sys.path.insert(0, ROOT)
    import bench

    s = bench.ClockSampler(0)
    s.start()
    rec = s.stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]
