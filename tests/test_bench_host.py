"""Host-side logic of bench.py (no GPU): the FP32-vs-FP64 error measures, the
clock record taken from nvidia-smi samples, the algorithmic byte count and the
oracle's CPU-baseline sampler."""
import datetime
import os
import time

import numpy as np
import pytest

import bench


def test_loglik_errors():
    l64 = np.array([-100.0, 2.0, 50.0])
    l32 = np.array([-100.001, 2.001, 50.0])
    n = np.array([1000, 100, 10])
    e = bench.loglik_errors(l32, l64, n)
    assert e["n_rows"] == 3
    assert e["max_rel_err"] == pytest.approx(5e-4)                  # 0.001 / 2
    assert e["n_rows_rel_above_1e-4"] == 1
    # max(|L|, 0.1 N): 100 for the first row, max(2, 10) = 10 for the second
    assert e["max_err_over_max_L_0p1N"] == pytest.approx(1e-4)
    assert e["max_abs_err_per_meas"] == pytest.approx(1e-5)
    assert e["max_abs_err"] == pytest.approx(1e-3)


def test_alg_bytes_per_meas():
    # two passes over 22 B of inputs plus a 27-float state written and read
    # every ck events (two events per measurement)
    assert bench.alg_bytes_per_meas(64) == pytest.approx(44 + 2 * 4 * 27 * 2 / 64)


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler_with(rows, window, tmp_path):
    s = bench.ClockSampler(0)
    path = tmp_path / "clocks.csv"
    with open(path, "w") as f:
        for ts, mhz, reasons in rows:
            stamp = datetime.datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
            flags = ["Active" if r in reasons else "Not Active"
                     for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                               "sw_power_cap")]
            f.write(", ".join([stamp, "0", str(mhz), "2070", "900.0", "0x0"] + flags) + "\n")
    s.proc = _FakeProc()
    s.path = str(path)
    s.mark(*window)
    # stop() waits (bounded) for one more sample than the file holds
    s._wait_lines = lambda n, limit_s: None
    return s


def test_clock_samples_inside_the_timed_window(tmp_path):
    t0 = time.time()
    rows = [(t0 - 1.0, 1000, set()), (t0 + 0.1, 2070, set()), (t0 + 0.2, 2060, {"sw_power_cap"}),
            (t0 + 5.0, 900, {"hw_slowdown"})]
    clk = _sampler_with(rows, (t0, t0 + 0.3), tmp_path).stop()
    assert clk["samples_from"] == "timed window" and clk["samples"] == 2
    assert clk["sm_mhz"] == pytest.approx(2065.0)
    assert clk["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(tmp_path / "clocks.csv")


def test_clock_samples_nearest_a_short_window(tmp_path):
    t0 = time.time()
    rows = [(t0 - 2.0, 1500, set()), (t0 - 0.5, 2070, set()), (t0 + 0.6, 2070, {"hw_slowdown"})]
    clk = _sampler_with(rows, (t0, t0 + 0.001), tmp_path).stop()
    assert clk["samples_from"] == "nearest to the timed window" and clk["samples"] == 2
    assert clk["reasons"] == ["hw_slowdown"]


def test_oracle_sample_rate_single_series():
    import synth
    wl = synth.c1()
    rate, cores, desc = bench.oracle_sample_rate(wl, 0.3, 4, 100, grad=False)
    assert rate > 0 and cores == 1                 # one series, one set: one core
    assert "closed forms" in desc and "first 100 measurements" in desc
