"""Host-side pieces of the measurement tools that need no GPU: the clock
sampler's parsing of nvidia-smi rows, the rule that rejects a timed region's
clocks, and the profiling commands quoted in the ncu summaries."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

# Rows as `nvidia-smi --format=csv,noheader,nounits` prints the sampler's
# fields: SM clock, max SM clock, power, active-reason mask, then hw_slowdown,
# hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap.
CLEAN = "2070, 2070, 812.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
CAPPED = "1905, 2070, 1398.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
THERMAL = "1500, 2070, 1390.00, 0x0000000000000020, Not Active, Not Active, Active, Not Active"
LOCKED = "1200, 2070, 600.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"


def _summary(rows):
    s = bench.ClockSampler(0)
    s.lines = list(rows)
    return s.summary()


def test_summary_takes_the_median_clock_and_collects_reasons():
    c = _summary([CLEAN, CLEAN, CAPPED, "garbage", "", "[N/A], 2070, 0, 0x0, a, b, c, d"])
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_summary_without_samples():
    c = _summary([])
    assert c["samples"] == 0 and c["sm_mhz"] is None and c["reasons"] == []
    assert bench.clock_verdict(c) is None


def test_clean_and_power_capped_runs_are_kept():
    assert bench.clock_verdict(_summary([CLEAN] * 5)) is None
    # The power cap lowers the clock for a reason: kept and noted.
    assert bench.clock_verdict(_summary([CAPPED] * 5)) is None


def test_thermal_slowdown_is_rejected():
    why = bench.clock_verdict(_summary([CLEAN, THERMAL, CLEAN]))
    assert why is not None and "sw_thermal_slowdown" in why


def test_clock_held_low_with_no_reason_is_rejected():
    why = bench.clock_verdict(_summary([LOCKED] * 4))
    assert why is not None and "no reason" in why
    # One low sample does not move the median.
    assert bench.clock_verdict(_summary([CLEAN, CLEAN, LOCKED])) is None


def test_hardware_slowdown_is_rejected_even_at_full_clock():
    row = "2070, 2070, 900.00, 0x0000000000000008, Active, Not Active, Not Active, Not Active"
    assert "hw_slowdown" in bench.clock_verdict(_summary([row]))


def test_profile_commands_in_profiles_parse_to_valid_problems():
    # Every profiling command that a summary under profiles/ gives must still
    # be accepted by the CLI and describe a problem the library accepts.
    import glob
    import re
    import shlex

    import paper_1502_07028_gb300 as P
    from paper_1502_07028_gb300 import profile_sweep

    found = 0
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(path).read().replace("\\\n", " ")
        for m in re.finditer(r"python -m paper_1502_07028_gb300\.profile_sweep([^\n`]*)", text):
            a = profile_sweep.parser().parse_args(shlex.split(m.group(1)))
            stages = P.ptca_schedule(profile_sweep.config(a))
            assert sum(len(s) for s in stages) == profile_sweep.config(a).N
            found += 1
        for m in re.finditer(r"python bench\.py([^\n`]*)", text):
            bench.parser().parse_args(shlex.split(m.group(1)))
            found += 1
    assert found >= 4


def test_every_ncu_command_in_profiles_leaves_the_clocks_alone():
    # An ncu run locks the GPU clocks unless told not to; every capture
    # command quoted under profiles/ must carry --clock-control none.
    import glob
    import re

    n = 0
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(path).read().replace("\\\n", " ")
        for m in re.finditer(r"^\s*ncu (?=-)(?!-i )[^\n]*", text, re.M):
            assert "--clock-control none" in m.group(0), (path, m.group(0))
            n += 1
    assert n >= 3
