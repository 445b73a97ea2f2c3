"""CPU checks of bench.py's host-side bookkeeping: the algorithmic byte counts
per phase, the clock sampler's timed-region filter and throttle-reason parsing,
and the committed DRAM-traffic lines it reads."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_per_phase(bench):
    n = 512
    N = M = n ** 3
    b = bench.algorithmic_bytes(n, n, 6)
    # interpolation: read disp, vel (24 N) + 3 force components (12 M), write disp, vel (24 N)
    assert b["interp_kick_drift"] == 48 * N + 12 * M
    # deposit: 24 N on the first of 6 steps, 12 N on the other 5, density written once
    assert b["deposit"] == pytest.approx((24 + 5 * 12) / 6 * N + 4 * M)
    assert b["fft_y_fwd"] == b["fft_y_inv"] == 8 * M
    assert b["grad_stencil"] == 16 * M
    # the forward x pass clears the consumed density on all but the last step
    assert b["fft_x_fwd"] == pytest.approx(8 * M + 4 * M * 5 / 6)


def test_clock_sampler_keeps_only_the_timed_region(bench):
    cs = bench.ClockSampler(0)
    line = "0, {sm}, 2070, 900.5, 0x0, Not Active, Not Active, {swt}, {pc}"
    cs.lines = [(1.0, line.format(sm=1000, swt="Not Active", pc="Not Active")),    # warm-up
                (2.0, line.format(sm=2070, swt="Not Active", pc="Active")),
                (2.1, line.format(sm=2060, swt="Not Active", pc="Not Active")),
                (2.2, line.format(sm=2070, swt="Not Active", pc="Not Active")),
                (9.0, line.format(sm=500, swt="Active", pc="Not Active"))]        # after
    cs.window = (1.5, 3.0)
    # a stand-in for the nvidia-smi process and reader thread that have ended
    cs.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    cs.t = type("T", (), {"join": lambda self, timeout=None: None})()
    info = cs.stop()
    assert info["samples"] == 3
    assert info["sm_mhz"] == 2070.0
    assert info["sm_max_mhz"] == 2070.0
    assert info["reasons"] == ["sw_power_cap"]


def test_clock_sampler_reports_an_empty_region(bench):
    cs = bench.ClockSampler(0)
    cs.lines = [(1.0, "0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active")]
    cs.window = (5.0, 6.0)
    cs.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    cs.t = type("T", (), {"join": lambda self, timeout=None: None})()
    assert cs.stop()["sm_mhz"] is None


def test_traffic_lines_parse(bench):
    # each committed TRAFFIC line is either current (an integer byte count of the
    # right magnitude) or dropped because its kernel source changed
    for k in ("interp_kick_drift", "deposit", "grad_stencil", "fft_z_green"):
        v = bench.measured_traffic(k)
        assert v is None or 5e8 < v < 2e10
    assert bench.measured_traffic("no_such_kernel") is None


def test_cufft_comparison_runs_and_reports_failures(bench):
    import torch
    r = bench.cufft_comparison(16, torch.device("cpu"), reps=1)
    assert r["mesh"] == 16 and r["ms_rfftn_green_irfftn"] > 0
    # a failure is reported in the line instead of ending the benchmark
    assert "error" in bench.cufft_comparison(-1, torch.device("cpu"), reps=1)
