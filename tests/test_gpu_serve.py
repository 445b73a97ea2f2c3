"""Continuous-batching server (batched DKD steps with per-slot coefficients,
captured CUDA graphs, slots admitted and retired between steps): every result
must equal the same request run alone (the kernels are the same; only the
order of float atomics in the deposit differs), and no request is lost."""
import pytest
import torch

from paper_2510_05206_gb300 import serve

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _alone(r):
    c = serve.SizeClass(r.n, 1, DEV, use_graph=False)
    c.admit(serve.Request(r.rid, r.n, r.n_steps, r.seed, 0.0), 0, 0.0)
    while c.active():
        c.launch_step()
        c.pending.synchronize()
        c.step_done()
    torch.cuda.synchronize()
    out = c.host_disp[0].clone()
    c.pm.close()
    return out


@pytest.mark.parametrize("use_graph", [True, False])
def test_each_result_same_alone_and_in_the_mix(use_graph):
    reqs = serve.make_stream(14, sizes=(32, 64), steps=(2, 5), rate=400.0, seed=3)
    # few slots: requests queue, slots are reused, different step indices share launches
    done, wall = serve.serve(reqs, device=DEV, slots={32: 3, 64: 2}, use_graph=use_graph, keep_results=True)
    assert sorted(r.rid for r in done) == list(range(14))
    for r in done:
        assert r.done >= r.admitted >= r.arrival
        alone = _alone(r)
        rms = torch.sqrt((alone ** 2).sum(0).mean())
        assert float((r.result - alone).abs().max() / rms) < 1e-5, r.rid


def test_budget_admission_single_slot():
    reqs = serve.make_stream(5, sizes=(32,), steps=(2, 3), rate=1000.0, seed=4)
    slots = serve.slots_for_budget([32], budget_bytes=1.0)     # nothing fits: one slot minimum
    assert slots == {32: 1}
    done, wall = serve.serve(reqs, device=DEV, slots=slots)
    assert sorted(r.rid for r in done) == list(range(5))
    st = serve.latency_stats(done, wall)
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_sequential_baseline_matches_server():
    reqs = serve.make_stream(4, sizes=(32,), steps=(2, 3), rate=1000.0, seed=5)
    done, wall = serve.serve_sequential(reqs, device=DEV)
    assert all(r.done > 0 for r in done)
