"""CPU checks of the serving loop's host logic: the seeded Poisson request
stream, admission by HBM budget (slots per size class from the library's
workspace sizing), and the latency statistics."""
import numpy as np
import pytest

from paper_2510_05206_gb300 import build, serve
from paper_2510_05206_gb300.pm import workspace_bytes


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_request_stream_is_seeded_and_well_formed():
    a = serve.make_stream(400, sizes=(64, 128, 256), steps=(4, 10), rate=200.0, seed=8)
    b = serve.make_stream(400, sizes=(64, 128, 256), steps=(4, 10), rate=200.0, seed=8)
    assert [(r.n, r.n_steps, r.seed, r.arrival) for r in a] == [(r.n, r.n_steps, r.seed, r.arrival) for r in b]
    t = np.array([r.arrival for r in a])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert {r.n for r in a} == {64, 128, 256}
    assert {r.n_steps for r in a} <= set(range(4, 11)) and len({r.n_steps for r in a}) == 7
    # exponential gaps of mean 1/rate (399 gaps: within 4 standard errors)
    gaps = np.diff(t)
    assert abs(gaps.mean() * 200.0 - 1.0) < 4.0 / np.sqrt(len(gaps))
    assert len({r.rid for r in a}) == 400


def test_slots_fit_the_budget_share():
    sizes = [64, 128, 256]
    for budget in (2e9, 8e9, 64e9):
        slots = serve.slots_for_budget(sizes, budget)
        share = budget / len(sizes)
        for n, cap in zip(sizes, (32, 16, 4)):
            per = workspace_bytes(serve.class_config(n, 1)) + 2 * 3 * 4 * n ** 3
            assert 1 <= slots[n] <= cap
            assert slots[n] == 1 or slots[n] * per <= share
            # the largest count that fits (or the cap)
            assert slots[n] == cap or (slots[n] + 1) * per > share or slots[n] == 1


def test_slots_grow_with_the_budget():
    sizes = [64, 128, 256]
    small = serve.slots_for_budget(sizes, 1e9)
    large = serve.slots_for_budget(sizes, 100e9)
    assert all(small[n] <= large[n] for n in sizes)
    assert large == {64: 32, 128: 16, 256: 4}


def test_latency_stats():
    reqs = [serve.Request(i, 64, 4, i, arrival=0.1 * i) for i in range(10)]
    for i, r in enumerate(reqs):
        r.done = r.arrival + 0.010 * (i + 1)
    st = serve.latency_stats(reqs, wall=2.0)
    assert st["requests"] == 10 and st["requests_per_s"] == 5.0
    assert st["p50_ms"] == pytest.approx(55.0)
    assert st["mean_ms"] == pytest.approx(55.0)
    assert st["p99_ms"] == pytest.approx(99.1)
