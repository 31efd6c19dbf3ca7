"""The benchmark's clock record on the CPU: nvidia-smi samples (csv, no
header, no units) summarised as the median SM clock, the maximum clock and
every throttle reason seen active; the sampler's stop() on a canned file."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

IDLE = "0, 2070, 2070, 250.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"


def sample(mhz, power_cap=False, thermal=False):
    return (f"0, {mhz}, 2070, 1190.5, 0x0000000000000004, Not Active, Not Active, "
            f"{'Active' if thermal else 'Not Active'}, {'Active' if power_cap else 'Not Active'}\n")


def test_median_and_no_reasons():
    s = bench.parse_clock_samples([sample(1965), sample(2070), IDLE, sample(2010), sample(2070)])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}
    s = bench.parse_clock_samples([sample(1800), sample(1900), sample(2000)])
    assert s["sm_mhz"] == 1900.0


def test_reasons_seen_in_any_sample():
    s = bench.parse_clock_samples([sample(2070), sample(1700, power_cap=True), sample(1500, thermal=True)])
    assert s["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]


def test_unreadable_lines_are_skipped():
    lines = ["", "garbage\n", "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
             "0, 1.2.3, 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n", sample(2040)]
    s = bench.parse_clock_samples(lines)
    assert s["samples"] == 1 and s["sm_mhz"] == 2040.0
    assert bench.parse_clock_samples(["garbage\n"]) is None
    assert bench.parse_clock_samples([]) is None


def test_sampler_stop_reads_and_removes_its_file(tmp_path):
    class Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0
    path = tmp_path / "clocks.csv"
    path.write_text(sample(2070) + sample(2070, power_cap=True) + sample(1980))
    s = bench.ClockSampler(0)
    s.proc, s.path = Proc(), str(path)
    out = s.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not path.exists()
    assert bench.ClockSampler(0).stop() is None        # never started (no nvidia-smi): no record
