"""Continuous-batching server for PM simulation requests (batched BullFrog
steps, Sec. 2.4-2.5, over slots of same-size simulations).

Requests of different mesh sizes and step counts arrive over time.  Each size
class owns one libpmgb handle with a fixed number of slots (chosen from the HBM
budget at start), its own CUDA stream, and a CUDA graph of one batched DKD step
over all its slots (``pm_step_slots``); every slot reads its own step
coefficients, so slots at different step indices and with different step
counts share every launch, and idle slots are skipped by the kernels.  Between
steps the host retires finished slots (their final state is copied to pinned
host memory), admits queued requests into free slots (Zel'dovich ICs for that
slot only), and uploads the per-slot coefficients.  Size classes run on
separate streams, so their work overlaps on the device.

Latency of a request = time from its arrival to the moment its result (final
displacements and velocities) is in host memory.
"""
import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import pm as pmmod


@dataclass
class Request:
    rid: int
    n: int              # particles (= mesh cells) per dimension
    n_steps: int
    seed: int
    arrival: float      # seconds after the start of the stream
    admitted: float = -1.0
    done: float = -1.0
    result: object = None   # final displacements (host), kept when serve(..., keep_results=True)


def make_stream(n_req, sizes=(64, 128, 256), steps=(4, 10), rate=100.0, seed=8):
    """Seeded Poisson arrival stream: sizes uniform over `sizes`, step counts
    uniform in [steps[0], steps[1]], exponential inter-arrival times of mean 1/rate."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_req))
    t -= t[0]
    return [Request(i, int(rng.choice(sizes)), int(rng.integers(steps[0], steps[1] + 1)),
                    int(rng.integers(1 << 30)), float(t[i])) for i in range(n_req)]


def class_config(n, batch, **kw):
    """Size class: L = 2 Mpc/h per cell, particles = mesh cells, CIC, BullFrog."""
    base = dict(n_part=n, n_mesh=n, box=2.0 * n, batch=batch, n_steps=10)
    base.update(kw)
    return pmmod.Config(**base)


def _noise(n, seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randn(n ** 3, generator=g, device=device, dtype=torch.float32)


class SizeClass:
    def __init__(self, n, slots, device, use_graph=True, keep_results=False):
        self.keep = keep_results
        self.n = n
        self.B = slots
        self.device = device
        self.stream = torch.cuda.Stream(device=device)
        self.copy_stream = torch.cuda.Stream(device=device)   # result copies overlap the next steps
        with torch.cuda.stream(self.stream):
            self.pm = pmmod.PM(class_config(n, slots), device=device)
            self.disp, self.vel = self.pm.new_state()
        N = n ** 3
        self.host_disp = torch.empty((slots, 3, N), dtype=torch.float32, pin_memory=True)
        self.host_vel = torch.empty((slots, 3, N), dtype=torch.float32, pin_memory=True)
        self.req = [None] * slots          # Request in each slot
        self.step = np.full(slots, -1, dtype=np.int32)
        self.nsteps = np.full(slots, 1, dtype=np.int32)
        self.pending = None                # event of the step in flight
        self.retiring = []                 # (event, request) copies in flight
        self.graph = None
        if use_graph:
            self._capture()

    def _capture(self):
        # warm up outside capture (first launches set kernel attributes), then capture one step
        with torch.cuda.stream(self.stream):
            self.pm.set_slots(self.nsteps, self.step)       # all idle: the kernels return at once
            self.pm.step_slots(self.disp, self.vel)
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self.pm.step_slots(self.disp, self.vel)
        self.graph = g

    def free_slots(self):
        return [i for i in range(self.B) if self.req[i] is None]

    def admit(self, r, slot, now):
        N = self.n ** 3
        with torch.cuda.stream(self.stream):
            noise = _noise(self.n, r.seed, self.device)
            self.pm.ic_zeldovich_slot(slot, noise, self.disp[slot], self.vel[slot])
        self.req[slot] = r
        self.step[slot] = 0
        self.nsteps[slot] = r.n_steps
        r.admitted = now

    def active(self):
        return any(q is not None and s >= 0 for q, s in zip(self.req, self.step))

    def launch_step(self):
        with torch.cuda.stream(self.stream):
            self.pm.set_slots(self.nsteps, self.step)
            if self.graph is not None:
                self.graph.replay()
            else:
                self.pm.step_slots(self.disp, self.vel)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        self.pending = ev

    def step_done(self):
        """Advance step counters after the step in flight finished; start the
        copies of finished slots.  Returns True if a step completed."""
        if self.pending is None or not self.pending.query():
            return False
        step_ev = self.pending
        self.pending = None
        for i in range(self.B):
            if self.req[i] is None or self.step[i] < 0:
                continue
            self.step[i] += 1
            if self.step[i] >= self.nsteps[i]:
                # the slot is idle for the kernels from now on (inactive coefficients), so its
                # state can be copied on the copy stream while the other slots keep stepping
                self.copy_stream.wait_event(step_ev)
                with torch.cuda.stream(self.copy_stream):
                    self.host_disp[i].copy_(self.disp[i], non_blocking=True)
                    self.host_vel[i].copy_(self.vel[i], non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(self.copy_stream)
                self.retiring.append((ev, self.req[i], i))
                self.step[i] = -1          # the slot stays held until its copy completes
        return True

    def collect(self, now):
        done = []
        keep = []
        for ev, r, i in self.retiring:
            if ev.query():
                r.done = now()
                if self.keep:
                    r.result = self.host_disp[i].clone()
                self.req[i] = None
                done.append(r)
            else:
                keep.append((ev, r, i))
        self.retiring = keep
        return done


def slots_for_budget(sizes, budget_bytes, max_slots=(32, 16, 4)):
    """Slots per size class: the largest counts (up to max_slots) whose state
    plus libpmgb workspace fit in an equal share of the HBM budget (admission
    control by device memory)."""
    out = {}
    share = budget_bytes / len(sizes)
    for n, cap in zip(sizes, max_slots):
        per = pmmod.workspace_bytes(class_config(n, 1)) + 2 * 3 * 4 * n ** 3 * 1.0
        out[n] = int(max(1, min(cap, share // per)))
    return out


def serve(requests, device="cuda", slots=None, use_graph=True, budget_bytes=None, poll_s=0.0002,
          keep_results=False):
    """Continuous batching over the request stream (arrival times honoured in
    real time).  Returns (requests with timestamps, wall seconds)."""
    sizes = sorted({r.n for r in requests})
    if slots is None:
        free, _ = torch.cuda.mem_get_info(device)
        slots = slots_for_budget(sizes, budget_bytes or 0.5 * free)
    classes = {n: SizeClass(n, slots[n], device, use_graph, keep_results) for n in sizes}
    queue = {n: deque() for n in sizes}
    torch.cuda.synchronize(device)
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    finished = []
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    while len(finished) < len(requests):
        t = now()
        while pending and pending[0].arrival <= t:
            r = pending.popleft()
            queue[r.n].append(r)
        progressed = False
        for n, c in classes.items():
            finished += c.collect(now)
            if c.pending is not None:
                progressed |= c.step_done()
            if c.pending is None:
                for slot in c.free_slots():
                    if not queue[n]:
                        break
                    c.admit(queue[n].popleft(), slot, now())
                if c.active():
                    c.launch_step()
                    progressed = True
        if not progressed and poll_s:
            time.sleep(poll_s)
    wall = now()
    for c in classes.values():
        c.pm.close()
    return finished, wall


def serve_sequential(requests, device="cuda"):
    """Baseline: one request at a time, in arrival order, each a batch-1 run
    (ICs, all steps, copy of the final state to host), same kernels."""
    sizes = sorted({r.n for r in requests})
    pms = {n: pmmod.PM(class_config(n, 1), device=device) for n in sizes}
    host = {n: (torch.empty((1, 3, n ** 3), dtype=torch.float32, pin_memory=True),
                torch.empty((1, 3, n ** 3), dtype=torch.float32, pin_memory=True)) for n in sizes}
    state = {n: pms[n].new_state() for n in sizes}
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    now = lambda: time.perf_counter() - t0
    for r in sorted(requests, key=lambda q: q.arrival):
        while now() < r.arrival:
            time.sleep(0.0002)
        pm = pms[r.n]
        d, v = state[r.n]
        r.admitted = now()
        noise = _noise(r.n, r.seed, device)
        pm.ic_zeldovich_slot(0, noise.reshape(1, -1), d, v)
        pm.set_slots([r.n_steps], [0])
        for s in range(r.n_steps):
            pm.set_slots([r.n_steps], [s])
            pm.step_slots(d, v)
        host[r.n][0].copy_(d, non_blocking=True)
        host[r.n][1].copy_(v, non_blocking=True)
        torch.cuda.current_stream(device).synchronize()
        r.done = now()
    wall = now()
    for p in pms.values():
        p.close()
    return list(requests), wall


def latency_stats(reqs, wall):
    lat = np.array([r.done - r.arrival for r in reqs])
    return {"requests": len(reqs), "requests_per_s": len(reqs) / wall, "wall_s": wall,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
