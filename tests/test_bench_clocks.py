"""The benchmark's clock sampler on the CPU: a stand-in nvidia-smi on PATH
prints the query's CSV rows; the sampler waits for the first row before the
timed region starts, keeps the rows printed during it, and reports the
median SM clock, the maximum clock and every throttle reason seen Active; it
says so when nvidia-smi is missing."""
import importlib.util
import os
import stat
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _fake_smi(tmp_path, rows):
    body = "".join(f'  echo "{r}"\n' for r in rows)
    script = tmp_path / "nvidia-smi"
    script.write_text("#!/bin/sh\nwhile true; do\n" + body + "  sleep 0.02\ndone\n")
    script.chmod(script.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def _sample(bench, monkeypatch, path_dir, seconds=0.3):
    monkeypatch.setenv("PATH", path_dir + os.pathsep + os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(seconds)
    out = s.stop()
    assert not os.path.exists(s.path) and s.out.closed
    return out


def test_median_clock_and_power_cap(bench, monkeypatch, tmp_path):
    d = _fake_smi(tmp_path, ["0, 1965, 2070, 812.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
                             "0, 2070, 2070, 700.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
                             "0, 2070, 2070, 705.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"])
    out = _sample(bench, monkeypatch, d)
    assert out["samples"] >= 3 and out["window"] == "timed region"
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_thermal_and_hardware_slowdowns_are_reported(bench, monkeypatch, tmp_path):
    d = _fake_smi(tmp_path, ["0, 1200, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active",
                             "garbage line that is not csv",
                             "0, [N/A], 2070, 1400.0, 0x0, Not Active, Not Active, Not Active, Not Active"])
    out = _sample(bench, monkeypatch, d)
    assert out["sm_mhz"] == 1200.0  # the unparsable rows are skipped
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_missing_nvidia_smi(bench, monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    out = s.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]
    assert not os.path.exists(s.path) and s.out.closed


def _script(tmp_path, body):
    script = tmp_path / "nvidia-smi"
    script.write_text("#!/bin/sh\n" + body)
    script.chmod(script.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def test_rows_before_the_timed_region_are_left_out(bench, monkeypatch, tmp_path):
    """The first row (idle clock) is out before start() returns; the rows
    that follow (clock under load) are the ones reported."""
    d = _script(tmp_path, 'echo "0, 345, 2070, 90.0, 0x1, Not Active, Not Active, Not Active, Not Active"\n'
                          'sleep 0.2\nwhile true; do\n'
                          '  echo "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"\n'
                          '  sleep 0.02\ndone\n')
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    s.start()
    assert s.skip == 1
    time.sleep(0.5)
    out = s.stop()
    assert out["window"] == "timed region" and out["sm_mhz"] == 2070.0 and out["samples"] >= 3


def test_a_sampler_that_prints_late_or_never_is_bounded(bench, monkeypatch, tmp_path):
    d = _script(tmp_path, "exec sleep 5\n")
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    t0 = time.time()
    s.start(ready_timeout=0.3)
    assert time.time() - t0 < 2.0
    out = s.stop()
    assert out["sm_mhz"] is None and out["samples"] == 0 and out["window"] == "just before the timed region"


def test_only_rows_before_the_region_are_reported_as_such(bench, monkeypatch, tmp_path):
    d = _script(tmp_path, 'echo "0, 1980, 2070, 600.0, 0x0, Not Active, Not Active, Not Active, Not Active"\n'
                          "exec sleep 5\n")
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    s.start()
    out = s.stop()
    assert out["window"] == "just before the timed region" and out["sm_mhz"] == 1980.0
