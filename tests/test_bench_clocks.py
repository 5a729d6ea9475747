"""The benchmark's clock sampler on the CPU: a stand-in nvidia-smi on PATH
prints the query's CSV rows; the sampler reports the median SM clock, the
maximum clock and every throttle reason seen Active, and says so when
nvidia-smi is missing."""
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
    assert out["samples"] >= 3
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



def test_a_sampler_that_never_prints_reports_no_clock(bench, monkeypatch, tmp_path):
    script = tmp_path / "nvidia-smi"
    script.write_text("#!/bin/sh\nexec sleep 5\n")
    script.chmod(script.stat().st_mode | stat.S_IXUSR)
    out = _sample(bench, monkeypatch, str(tmp_path), seconds=0.1)
    assert out["sm_mhz"] is None and out["samples"] == 0 and out["reasons"] == []
