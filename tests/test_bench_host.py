"""Host-side pieces of bench.py that need no GPU: the clock sampler's summary
of nvidia-smi lines (median SM clock under load, maximum clock, the throttle
reasons seen) and the launcher check of --gpus against WORLD_SIZE."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def summary(lines):
    cs = bench.ClockSampler()
    cs.samples = [[v.strip() for v in ln.split(",")] for ln in lines]
    return cs.stop()


def test_clock_summary_median_max_and_reasons():
    lines = [
        "2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1965, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2010, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",     # unreadable sample
        "2070, 2070",                                                  # truncated line
    ]
    s = summary(lines)
    assert s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_slowdowns_and_handles_no_samples():
    s = summary(["1400, 2070, 800, 0x08, Active, Not Active, Active, Not Active"])
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert summary([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_gpus_flag_must_match_the_launcher():
    # without torchrun WORLD_SIZE is 1, so --gpus 2 is refused with status 2 before any GPU work
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2"], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 2
