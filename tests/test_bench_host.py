"""Host-side logic of bench.py, on CPU.

* The clock sampler reads the CSV lines of the GPU-query tool (a fake on PATH here): it keeps the
  rows of its own GPU, skips malformed ones, reports the median SM clock under load, the largest
  maximum clock and every throttle reason seen active; without the tool it reports nothing.
* The tensor-core roofline takes the GEMM leg with the longer device time and divides the MMA
  flops it issued by that time, against the BF16 peak it is given.
"""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

ROWS = [
    "GPU-a, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
    "GPU-b, 1000, 2070, 300.0, 0x0, Active, Not Active, Not Active, Not Active",   # another GPU
    "GPU-a, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
    "garbage line",
    "GPU-a, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
]


def _fake_tool(tmp_path, rows):
    path = tmp_path / "nvidia-smi"
    body = "".join("echo '%s'\n" % r for r in rows)
    path.write_text("#!/bin/sh\n" + body + "exec sleep 30\n")
    path.chmod(path.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def test_clock_sampler_reads_its_gpu(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_tool(tmp_path, ROWS) + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(uuid="GPU-a")
    c.start()
    assert c.p is not None
    t0 = time.time()
    while time.time() - t0 < 10 and os.path.getsize(c.f.name) < sum(len(r) + 1 for r in ROWS):
        time.sleep(0.05)
    out = c.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_sampler_all_gpus_and_slowdown(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_tool(tmp_path, ROWS) + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler()
    c.start()
    t0 = time.time()
    while time.time() - t0 < 10 and os.path.getsize(c.f.name) < sum(len(r) + 1 for r in ROWS):
        time.sleep(0.05)
    out = c.stop()
    assert out["samples"] == 4 and out["sm_mhz"] == 2025.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_sampler_without_tool(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))   # an empty directory: no query tool
    c = bench.ClockSampler()
    c.start()
    assert c.p is None and c.stop() is None
    os.unlink(c.f.name)


def test_tc_roofline_takes_the_longer_leg():
    s = {"ms_gemm_chi0": 200.0, "flop_exec_gemm_chi0": 4.0e13, "n_gemm_chi0": 480,
         "ms_gemm_ec": 250.0, "flop_exec_gemm_ec": 6.0e13, "n_gemm_ec": 144}
    r = bench.tc_roofline(s, {"bf16_tflops": 2000.0, "bf16_tflops_sustained": 1700.0}, "measured")
    assert r["kernel"] == "k_ozgemm (ln det GEMMs)" and r["launches"] == 144
    assert r["achieved"] == pytest.approx(6.0e13 / 0.25 / 1e12)
    assert r["frac"] == pytest.approx(240.0 / 2000.0) and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    s["ms_gemm_ec"] = 0.0
    s["ms_gemm_chi0"] = 0.0
    assert bench.tc_roofline(s, {"bf16_tflops": 2000.0}, "measured") is None


def test_job_value_is_all_units_over_the_slowest_rank():
    assert bench.job_value(3, 4, 2.0) == 6.0
