"""Host logic of bench.py (CPU only): the clock record keeps only the nvidia-smi samples inside
the timed region's wall-clock window and reports the throttle reasons seen there."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Exited:
    """Stands in for the finished nvidia-smi process."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _line(ts, sm, smax=2070, slow="Not Active", power_cap="Not Active"):
    stamp = ts.strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{stamp}, 0, {sm}, {smax}, 900.5, 0x0, {slow}, Not Active, Not Active, {power_cap}\n"


def _sampler(lines, window):
    clk = bench.ClockSampler(0)
    clk.p = _Exited()
    clk.f.write("".join(lines))
    clk.f.flush()
    if window:
        clk.mark(*window)
    return clk.stop()


def test_only_samples_inside_the_timed_window_count():
    t0 = datetime.datetime(2026, 12, 3, 12, 0, 0)
    lines = [_line(t0 - datetime.timedelta(seconds=1), 1200, slow="Active"),     # warm-up: ignored
             _line(t0 + datetime.timedelta(milliseconds=100), 2070),
             _line(t0 + datetime.timedelta(milliseconds=200), 2055, power_cap="Active"),
             _line(t0 + datetime.timedelta(milliseconds=300), 2070),
             _line(t0 + datetime.timedelta(seconds=2), 900)]                      # after: ignored
    c = _sampler(lines, (t0, t0 + datetime.timedelta(milliseconds=400)))
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_reasons_inside_the_window_are_reported_and_malformed_lines_skipped():
    t0 = datetime.datetime(2026, 12, 3, 12, 0, 0)
    lines = ["not a sample\n",
             _line(t0 + datetime.timedelta(milliseconds=10), 1500, slow="Active"),
             "2026/12/03 12:00:00.020, 0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active\n"]
    c = _sampler(lines, (t0, t0 + datetime.timedelta(milliseconds=50)))
    assert c["samples"] == 1 and c["sm_mhz"] == 1500.0
    assert c["reasons"] == ["hw_slowdown"]


def test_without_nvidia_smi_the_record_says_so():
    clk = bench.ClockSampler(0)
    c = clk.stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]
    assert not os.path.exists(clk.f.name)


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle on the host cores, one solve per step) prints one
    JSON line with the contract's keys, the oracle as its cpu_baseline and a zero-copy e2e."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "tau00 solves/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "S=7" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]
