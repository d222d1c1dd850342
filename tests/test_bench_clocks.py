"""The benchmark's clock record (sampled with nvidia-smi during the timed region) on a fake
sample file: the median SM clock, the maximum, and every throttle reason seen active, so that a
run under thermal or hardware slowdown says so."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.proc = _DoneProcess()
    return s


def test_clean_run():
    rec = _sampler(["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active"] * 4).stop()
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 4}


def test_reasons_and_median():
    rec = _sampler([
        "0, 2070, 2070, 1300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1500, 2070, 1390.0, 0x40, Not Active, Active, Not Active, Not Active",
        "garbage line",
        "0, 2010, 2070, 1380.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]).stop()
    assert rec["samples"] == 4
    assert rec["sm_mhz"] == 1995.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_no_samples_and_no_tool():
    assert _sampler(["not a sample"]).stop() is None
    s = bench.ClockSampler(0)
    assert s.stop() is None                      # never started (no nvidia-smi): no record
