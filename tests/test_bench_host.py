"""Host-side parts of bench.py that need no GPU: the roofline arithmetic and the clock sampler."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synthetic  # noqa: E402


def test_cost_model_and_algorithmic_bytes_of_the_headline():
    # Section 2's cost model at p = 7: 7 * 8^3 reads and 12 * 8^4 + 15 * 8^3 flops per element
    assert bench.cost_per_element(7) == (3584, 56832)
    m = synthetic.cube_mesh(64, 7, seed=0)
    per_dof = {qb: bench.algorithmic_bytes(m, qb) / m.n_ldof for qb in (8, 4, 2)}
    # x and y once (16 B) + 6 factors per point + the int32 restriction, per L-vector node
    assert per_dof[8] == pytest.approx(93.1, abs=0.05)
    assert per_dof[4] == pytest.approx(57.5, abs=0.05)
    assert per_dof[2] == pytest.approx(39.7, abs=0.05)
    geo = bench.algorithmic_bytes(m, 4, geo=True)
    assert geo == 16 * m.n_ldof + (24 * 4 + 4 * 512) * m.n_elem + 4 * 512 * m.n_elem


def _fake_smi(tmp_path, startup_s, line):
    script = tmp_path / "nvidia-smi"
    script.write_text("#!%s\nimport sys, time\ntime.sleep(%r)\nwhile True:\n    print(%r, flush=True)\n"
                      "    time.sleep(0.05)\n" % (sys.executable, startup_s, line))
    script.chmod(script.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def test_clock_sampler_waits_for_a_slow_start(tmp_path, monkeypatch):
    # a sampler that starts after the region would report nothing: the fake tool needs 0.5 s to
    # print its first line, the region lasts 0.4 s
    d = _fake_smi(tmp_path, 0.5, "2070, 2070, 950.0, Not Active, Not Active, Not Active, Active")
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ.get("PATH", ""))
    with bench.ClockSampler(0) as clk:
        time.sleep(0.4)
    s = clk.summary()
    assert s["samples"] >= 2
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_sampler_reports_throttling(tmp_path, monkeypatch):
    d = _fake_smi(tmp_path, 0.0, "1500, 2070, 1400.0, Active, Not Active, Active, Not Active")
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ.get("PATH", ""))
    with bench.ClockSampler(0) as clk:
        time.sleep(0.3)
    s = clk.summary()
    assert s["sm_mhz"] == 1500.0 and s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_the_tool(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    with bench.ClockSampler(0, first_sample_s=0.5) as clk:
        time.sleep(0.05)
    assert clk.summary()["reasons"] == ["unavailable"]
