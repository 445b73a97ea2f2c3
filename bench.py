#!/usr/bin/env python
"""Benchmark: 512^3-particle PM simulations (512^3 mesh, L = 1000 Mpc/h, CIC,
6 BullFrog steps a = 0.02 -> 1), reported as PM particle-steps per second.

One bench step = one full simulation: Zel'dovich ICs from resident white noise,
6 DKD steps, and the final binned P(k) (FP64 bins read back to the host).
value = N * 6 * K / (time of K steps) summed over ranks (replicas: every rank
runs its own simulation; there is no data-path collective).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "512^3 PM particle-steps/s & %HBM roofline; batched serving p50/p99 latency"
UNIT = "particle-steps/s"
WORKLOAD = dict(workload="pm_512cubed_6step", n_part=512, n_mesh=512, box_mpc_h=1000.0, mass_assignment="CIC",
                stepper="bullfrog", n_steps=6, a_ini=0.02, a_end=1.0, grad_order=4, lap_order=0,
                pk_mesh=512, pk_bins=256, l2_policy="inputs larger than L2 (3.2 GB particle state, 3.7 GB workspace)")
NOISE_SEED = 3


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []            # (host time of arrival, csv line)
        self.window = (0.0, float("inf"))

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def begin(self):
        """Start of the timed region (the sampler runs from before the warm-up so that
        nvidia-smi's start-up latency does not eat the region)."""
        self.window = (time.perf_counter(), float("inf"))

    def end(self):
        self.window = (self.window[0], time.perf_counter())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if not self.window[0] <= ts <= self.window[1]:
                continue
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
                power.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples in the timed region"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    when the kernel's source changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic_pm_512cubed.md")
    csrc = os.path.join(ROOT, "paper_2510_05206_gb300", "csrc")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        p = ln.split()
        if len(p) == 5 and p[0] == "TRAFFIC" and p[1] == kernel:
            data = b"".join(open(os.path.join(csrc, f), "rb").read() for f in p[3].split("+"))
            if hashlib.sha256(data).hexdigest()[:16] == p[4]:
                return int(p[2])
            return None
    return None


def max_over_ranks(x, ws, dev):
    """The largest x over the ranks (the slowest rank's time sets the job's)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, seconds):
    """Units all ranks processed per second of the slowest rank (weak scaling:
    every rank runs its own replica of the workload)."""
    return units_per_rank * ws / seconds


def host_link_gbs(host):
    """Plain pinned-host <-> device copy rates of one state-sized buffer (context
    for the end-to-end number: the host link differs between machines)."""
    import torch
    dev_buf = torch.empty(host.shape, dtype=host.dtype, device="cuda")
    out = {}
    for name, (dst, src) in (("h2d", (dev_buf, host)), ("d2h", (host, dev_buf))):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        out[name] = 3 * host.numel() * host.element_size() / (e0.elapsed_time(e1) / 1e3) / 1e9
    del dev_buf
    return out


def cufft_comparison(n, dev, reps=10):
    """cuFFT (through torch.fft) on the spectral part of a PM step for comparison:
    real-to-complex 3D transform of an n^3 mesh, Poisson multiplier, complex-to-real
    back (the library's own passes do this as x, y forward, the fused z pass, y, x
    inverse).  Failures are reported in the line instead of ending the run."""
    import torch
    try:
        x = torch.randn(n, n, n, device=dev, dtype=torch.float32)
        kz = torch.fft.fftfreq(n, device=dev).view(n, 1, 1)
        ky = torch.fft.fftfreq(n, device=dev).view(1, n, 1)
        kx = torch.fft.rfftfreq(n, device=dev).view(1, 1, n // 2 + 1)
        k2 = kx ** 2 + ky ** 2 + kz ** 2
        k2[0, 0, 0] = 1.0
        green = (-1.0 / k2).to(torch.float32)
        green[0, 0, 0] = 0.0

        def chain():
            return torch.fft.irfftn(torch.fft.rfftn(x) * green, s=(n, n, n))

        for _ in range(3):
            chain()
        if torch.cuda.is_available() and x.is_cuda:
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                chain()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
        else:
            t0 = time.perf_counter()
            for _ in range(reps):
                chain()
            ms = (time.perf_counter() - t0) * 1e3 / reps
        del x, green, k2
        return {"mesh": n, "ms_rfftn_green_irfftn": ms}
    except Exception as e:  # noqa: BLE001 - a comparison must not end the benchmark
        return {"mesh": n, "error": f"{type(e).__name__}: {e}"}


def algorithmic_bytes(n_part, n_mesh, n_steps=6):
    """Compulsory HBM bytes per launch of each phase (float32; M = mesh cells,
    N = particles; complex half spectra count as M/2 complex = 4M bytes),
    averaged over the launches of one run of n_steps steps."""
    N, M = n_part ** 3, n_mesh ** 3
    later = (n_steps - 1) / n_steps          # share of the steps after the first
    return {
        # deposit: the first step of a run reads disp and vel (24 N), the later ones
        # the carried pre-drifted positions only (12 N); the density is written once (4 M)
        "deposit": (24 - 12 * later) * N + 4 * M,
        # read the real mesh, write the half spectrum; inside a run (all but the last
        # step) the consumed density is also cleared for the next deposit (4 M)
        "fft_x_fwd": 4 * M + 4 * M + 4 * M * later,
        "fft_y_fwd": 8 * M,                      # read + write half spectrum
        # finite-difference gradient (grad_order 2/4/6): the z pass maps the density
        # spectrum to the potential's, one inverse transform, then the stencil
        "fft_z_green": 4 * M + 4 * M,            # read 1 spectrum, write 1
        "fft_y_inv": 8 * M,                      # 1 spectrum in place
        "fft_x_inv": 4 * M + 4 * M,              # potential spectrum -> real potential
        "grad_stencil": 4 * M + 12 * M,          # read phi, write 3 components (float4 padding not counted)
        "interp_kick_drift": 48 * N + 12 * M,    # read disp, vel, 3 force components; write disp, vel
    }


def run_reference(args, ws, rank):
    """The oracle (FP64 numpy, as it stands) on the host cores: each step is one
    DKD step of a 128^3-particle sample of the same workload (128^3 mesh,
    L = 250 Mpc/h keeps the 1.95 Mpc/h cell)."""
    if rank != 0:
        return
    import numpy as np
    from oracle import cosmology, nbody
    from paper_2510_05206_gb300 import inputs

    n = 128
    cfg = nbody.Config(n_part=n, n_mesh=n, box=1000.0 * n / 512, n_steps=6)
    tab = cosmology.step_table(cfg.get_growth(), cfg.a_ini, cfg.a_end, cfg.n_steps)
    q = nbody.lattice(n, cfg.box)
    P, V = nbody.zeldovich_ic(cfg, inputs.white_noise(n, NOISE_SEED))
    for i in range(args.warmup):
        P, V = nbody.step(cfg, P, V, tab[i % 6], q)
    t0 = time.perf_counter()
    for i in range(args.steps):
        P, V = nbody.step(cfg, P, V, tab[i % 6], q)
    dt = time.perf_counter() - t0
    value = n ** 3 * args.steps / dt
    sample = f"{args.steps} DKD steps of a {n}^3-particle, {n}^3-mesh run (L = {cfg.box:g} Mpc/h), numpy FP64"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": WORKLOAD,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def host_cpu():
    """CPU model and logical core count of the host the oracle runs on."""
    model = platform.processor() or platform.machine()
    try:
        for ln in open("/proc/cpuinfo"):
            key = ln.split(":")[0].strip().lower()
            if key in ("model name", "cpu part", "hardware"):
                model = ln.split(":", 1)[1].strip()
                if key == "model name":
                    break
    except OSError:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count(), "machine": platform.machine()}


def cpu_baseline_sample():
    """Oracle timing on the host (rank 0, N = 1): ICs + 2 DKD steps at 128^3,
    and the 32^3 parity configuration in full."""
    import numpy as np
    from oracle import cosmology, nbody
    from paper_2510_05206_gb300 import inputs
    n = 128
    cfg = nbody.Config(n_part=n, n_mesh=n, box=1000.0 * n / 512, n_steps=6)
    tab = cosmology.step_table(cfg.get_growth(), cfg.a_ini, cfg.a_end, cfg.n_steps)
    q = nbody.lattice(n, cfg.box)
    w = inputs.white_noise(n, NOISE_SEED)
    t0 = time.perf_counter()
    P, V = nbody.zeldovich_ic(cfg, w)
    for i in range(2):
        P, V = nbody.step(cfg, P, V, tab[i], q)
    dt = time.perf_counter() - t0
    # the 32^3 parity configuration in full: ICs, 6 BullFrog steps and P(k) on the 32^3 mesh
    from oracle import mesh as omesh
    c1 = nbody.Config(n_part=32, n_mesh=32, box=256.0, n_steps=6)
    t1 = time.perf_counter()
    P1, V1 = nbody.zeldovich_ic(c1, inputs.white_noise(32, 1))
    P1, V1 = nbody.run(c1, P1, V1)
    omesh.power_spectrum(omesh.density_contrast(np.mod(nbody.lattice(32, 256.0) + P1, 256.0), 32, 256.0, 2),
                         256.0, 16)
    dt1 = time.perf_counter() - t1
    return {"value": n ** 3 * 2 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"Zel'dovich ICs + 2 DKD steps at {n}^3 particles / {n}^3 mesh, L = {cfg.box:g} Mpc/h "
                      f"(numpy FP64; {dt:.1f} s)",
            "threads_note": "numpy's FFT and scatter-add run on one thread, so OMP_NUM_THREADS = 1 and = nproc "
                            "time the same",
            "host": host_cpu(), "parity_config_32cubed_full_s": dt1}


def serving_benchmark(n_req, dev):
    """Continuous batching of a seeded Poisson stream of PM requests (sizes
    64^3 / 128^3 / 256^3 particles = mesh cells, L = 2 Mpc/h per cell, 4-10
    BullFrog steps), offered at the sequential service capacity, against the
    same stream served one request at a time on the same GPU."""
    from paper_2510_05206_gb300 import serve
    sizes, steps = (64, 128, 256), (4, 10)
    # sequential capacity: all requests of a calibration stream at t = 0
    cal = serve.make_stream(48, sizes, steps, rate=1e9, seed=18)
    serve.serve_sequential(cal[:6], device=dev)            # warm-up (first launches, tables)
    _, wall = serve.serve_sequential(cal, device=dev)
    capacity = len(cal) / wall
    cal = serve.make_stream(96, sizes, steps, rate=1e9, seed=19)
    _, wall_cb = serve.serve(cal, device=dev)
    cap_batched = len(cal) / wall_cb
    out = {"requests": n_req, "sizes": list(sizes), "steps": list(steps),
           "capacity_req_per_s": {"batched": cap_batched, "sequential": capacity},
           "note": "capacity: all requests at t = 0; loads: Poisson arrivals at the given multiple of the "
                   "sequential capacity; latency = arrival -> final state in host memory"}
    for mult in (1.0, 2.0):
        reqs = serve.make_stream(n_req, sizes, steps, rate=mult * capacity, seed=8)
        done, wall_b = serve.serve(reqs, device=dev)
        reqs = serve.make_stream(n_req, sizes, steps, rate=mult * capacity, seed=8)
        done_s, wall_s = serve.serve_sequential(reqs, device=dev)
        out[f"load_{mult:g}x"] = {"offered_rate_per_s": mult * capacity,
                                  "batched": serve.latency_stats(done, wall_b),
                                  "sequential": serve.latency_stats(done_s, wall_s)}
    return out


def adjoint_benchmark(dev, reps=5):
    """Gradient of the field-level chi^2 (128^3 particles on a 128^3 mesh,
    L = 500 Mpc/h, 10 BullFrog steps, CIC, sigma = 0.1 per cell) with respect to
    the white-noise field and sigma8: ICs + forward run + density, then the
    density VJP, the reverse adjoint of the 10 steps and the IC adjoint.
    Reports ms per gradient and the device memory the handle holds for 10 and
    for 40 steps (the adjoint stores no trajectory)."""
    import numpy as np
    import torch
    from paper_2510_05206_gb300 import PM, Config, workspace_bytes
    n, L, sigma = 128, 500.0, 0.1
    cfg = Config(n_part=n, n_mesh=n, box=L, n_steps=10)
    pm = PM(cfg, device=dev)
    rng = np.random.default_rng(NOISE_SEED + 4)
    noise = torch.from_numpy(rng.standard_normal((1, n ** 3), dtype=np.float32)).to(dev)
    target = torch.from_numpy(rng.standard_normal((1, n, n, n), dtype=np.float32)).to(dev) * sigma
    disp, vel = pm.new_state()
    adv = torch.empty_like(vel)

    def grad():
        pm.ic_zeldovich(noise, disp, vel)
        pm.run(disp, vel)
        dd = (pm.density(disp) - target) / sigma ** 2
        ad = pm.density_vjp(disp, dd)
        adv.zero_()
        pm.adjoint(disp, vel, ad, adv)
        return pm.ic_adjoint(noise, ad, adv)

    for _ in range(3):
        grad()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        grad()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / reps
    pm.close()
    ws10 = workspace_bytes(cfg)
    ws40 = workspace_bytes(Config(n_part=n, n_mesh=n, box=L, n_steps=40))
    return {"workload": "chi2_gradient_128cubed_on_128cubed_L500_10step_cic", "ms_per_gradient": ms,
            "gradients_per_s": 1e3 / ms, "particle_steps_per_s_fwd_plus_adj": n ** 3 * 10 * 2 / (ms / 1e3),
            "workspace_bytes_10_steps": ws10, "workspace_bytes_40_steps": ws40, "reps": reps}


def scaleup_benchmark(dev, reps=3):
    """One run of the scale-up configuration: 128^3 particles on a 256^3 mesh
    (L = 250 Mpc/h), TSC with interlacing, ICs + 10 BullFrog steps."""
    import numpy as np
    import torch
    from paper_2510_05206_gb300 import PM, Config
    n = 128
    pm = PM(Config(n_part=n, n_mesh=256, box=250.0, order=3, interlace=1, n_steps=10), device=dev)
    rng = np.random.default_rng(NOISE_SEED + 2)
    noise = torch.from_numpy(rng.standard_normal((1, n ** 3), dtype=np.float32)).to(dev)
    disp, vel = pm.new_state()
    for _ in range(3):
        pm.ic_zeldovich(noise, disp, vel)
        pm.run(disp, vel)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        pm.ic_zeldovich(noise, disp, vel)
        pm.run(disp, vel)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / reps
    pm.close()
    return {"workload": "pm_128cubed_on_256cubed_L250_tsc_interlaced_10step", "ms_per_run": ms,
            "ms_per_pm_step": ms / 10, "particle_steps_per_s": n ** 3 * 10 / (ms / 1e3)}


def jvp_benchmark(dev, reps=5):
    """Forward mode on the adjoint workload (128^3 / 128^3, L = 500, 10 steps):
    tangent ICs + the run with its tangent, and the P(k) tangent of the result."""
    import numpy as np
    import torch
    from paper_2510_05206_gb300 import PM, Config
    n = 128
    pm = PM(Config(n_part=n, n_mesh=n, box=500.0, n_steps=10), device=dev)
    rng = np.random.default_rng(NOISE_SEED + 5)
    w = torch.from_numpy(rng.standard_normal((1, n ** 3), dtype=np.float32)).to(dev)
    wt = torch.from_numpy(rng.standard_normal((1, n ** 3), dtype=np.float32)).to(dev)
    d, v = pm.new_state()
    td, tv = pm.new_state()

    def once():
        pm.ic_zeldovich(w, d, v)
        pm.ic_zeldovich(wt, td, tv)
        pm.jvp(d, v, td, tv)

    for _ in range(3):
        once()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        once()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / reps
    tp = time.perf_counter()
    for _ in range(reps):
        pm.power_spectrum_jvp(d, td, n, n // 2)
    ms_pk = (time.perf_counter() - tp) * 1e3 / reps
    pm.close()
    return {"workload": "jvp_128cubed_on_128cubed_L500_10step_cic", "ms_per_jvp_run": ms,
            "particle_steps_per_s_with_tangent": n ** 3 * 10 / (ms / 1e3), "ms_per_pk_jvp_host_timed": ms_pk}


def nufft_benchmark(dev, reps=3):
    """NUFFT force (ES kernel, width 5, grid upsampled twice, exact kernels) at
    256^3 particles with a 256^3 band (512^3 internal grid): ICs + 6 steps."""
    import numpy as np
    import torch
    from paper_2510_05206_gb300 import PM, Config
    n = 256
    pm = PM(Config(n_part=n, n_mesh=n, box=500.0, n_steps=6, grad_order=0, nufft=1), device=dev)
    rng = np.random.default_rng(NOISE_SEED)
    noise = torch.from_numpy(rng.standard_normal((1, n ** 3), dtype=np.float32)).to(dev)
    d, v = pm.new_state()
    for _ in range(2):
        pm.ic_zeldovich(noise, d, v)
        pm.run(d, v)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        pm.ic_zeldovich(noise, d, v)
        pm.run(d, v)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / reps
    pm.close()
    return {"workload": "pm_256cubed_nufft_band256_grid512_6step", "ms_per_run": ms, "ms_per_pm_step": ms / 6,
            "particle_steps_per_s": n ** 3 * 6 / (ms / 1e3)}


def lpt2_ic_benchmark(dev, reps=3):
    """2LPT initial conditions for the 512^3 lattice (four spectral chains and
    the source products) against the Zel'dovich ICs of the same handle size."""
    import numpy as np
    import torch
    from paper_2510_05206_gb300 import PM, Config
    n = WORKLOAD["n_part"]
    out = {"workload": f"ic_{n}cubed"}
    rng = np.random.default_rng(NOISE_SEED)
    noise = torch.from_numpy(rng.standard_normal((1, n ** 3), dtype=np.float32)).to(dev)
    for lpt in (1, 2):
        pm = PM(Config(n_part=n, n_mesh=WORKLOAD["n_mesh"], box=WORKLOAD["box_mpc_h"], lpt_order=lpt), device=dev)
        disp, vel = pm.new_state()
        for _ in range(3):
            pm.ic_zeldovich(noise, disp, vel)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            pm.ic_zeldovich(noise, disp, vel)
        t1.record()
        torch.cuda.synchronize()
        out["ms_2lpt" if lpt == 2 else "ms_zeldovich"] = t0.elapsed_time(t1) / reps
        pm.close()
        del disp, vel
    return out


def deconvolve_benchmark(dev, reps=3):
    """The 512^3 workload with the force density deconvolved by the squared mass
    assignment kernel (N_g = N with deconvolution), CIC and PCS: ICs + 6 BullFrog
    steps."""
    import numpy as np
    import torch
    from paper_2510_05206_gb300 import PM, Config
    n = WORKLOAD["n_part"]
    rng = np.random.default_rng(NOISE_SEED)
    noise = torch.from_numpy(rng.standard_normal((1, n ** 3), dtype=np.float32)).to(dev)
    out = {}
    for order, name in ((2, "cic"), (4, "pcs")):
        pm = PM(Config(n_part=n, n_mesh=WORKLOAD["n_mesh"], box=WORKLOAD["box_mpc_h"], n_steps=6, deconvolve=1,
                       order=order), device=dev)
        disp, vel = pm.new_state()
        for _ in range(2):
            pm.ic_zeldovich(noise, disp, vel)
            pm.run(disp, vel)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            pm.ic_zeldovich(noise, disp, vel)
            pm.run(disp, vel)
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / reps
        pm.close()
        del disp, vel
        out[name] = {"workload": f"pm_{n}cubed_6step_{name}_deconvolved", "ms_per_run": ms, "ms_per_pm_step": ms / 6,
                     "particle_steps_per_s": n ** 3 * 6 / (ms / 1e3)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--size", type=int, default=512, help="particles per dimension (512 = the benchmark workload)")
    ap.add_argument("--mesh", type=int, default=0, help="mesh cells per dimension (default = --size)")
    ap.add_argument("--no-serving", action="store_true", help="skip the continuous-batching measurement")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--no-extra", action="store_true", help="skip the adjoint and scale-up measurements")
    args = ap.parse_args()
    if args.size != 512 or (args.mesh and args.mesh != 512):
        # a reduced case for profiling captures; the config says so
        m = args.mesh or args.size
        WORKLOAD.update(workload=f"pm_{args.size}cubed_on_{m}cubed_6step_profiling_case", n_part=args.size,
                        n_mesh=m, box_mpc_h=1000.0 * m / 512, pk_mesh=m, pk_bins=m // 2)
    ws, rank, local = dist_env()

    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2510_05206_gb300 import PM, Config

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    n = WORKLOAD["n_part"]
    cfg = Config(n_part=n, n_mesh=WORKLOAD["n_mesh"], box=WORKLOAD["box_mpc_h"], order=2, n_steps=6,
                 a_ini=0.02, a_end=1.0, pk_mesh_max=WORKLOAD["pk_mesh"])
    pm = PM(cfg, device=dev)
    N = n ** 3
    rng = np.random.default_rng(NOISE_SEED + rank)
    noise_host = torch.from_numpy(rng.standard_normal(N, dtype=np.float32).reshape(1, N)).pin_memory()
    noise = noise_host.to(dev)
    disp, vel = pm.new_state()

    # one step of the workload: ICs, the run and the binned P(k) of the final state,
    # all enqueued without a host round trip (the P(k) bin sums stay on the device
    # and are turned into k, P(k) after the timed region)
    pk_sums = torch.zeros((1, WORKLOAD["pk_bins"]), dtype=torch.float64, device=dev)

    def one_sim():
        pm.ic_zeldovich(noise, disp, vel)
        pm.run(disp, vel)
        pm.power_spectrum_async(disp, pk_sums, WORKLOAD["pk_mesh"], WORKLOAD["pk_bins"])

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(max(args.warmup, 3)):
        one_sim()
    torch.cuda.synchronize()

    pm.profile(True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.begin()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        one_sim()
    t1.record()
    torch.cuda.synchronize()
    clocks.end()
    k, pk, cnt = pm.power_spectrum_finish(pk_sums, WORKLOAD["pk_mesh"], WORKLOAD["pk_bins"])
    if not (np.all(np.isfinite(pk)) and np.all(pk[cnt > 0] > 0)):
        raise RuntimeError("bench: the power spectrum of the final state is not finite and positive")
    clock_info = clocks.stop()
    ms = t0.elapsed_time(t1)
    prof = pm.profile_read()
    pm.profile(False)
    ms = max_over_ranks(ms, ws, dev)
    if ws > 1:
        dist.barrier()
    value = whole_job_rate(N * cfg.n_steps * args.steps, ws, ms / 1e3)

    # end to end through the host-buffer C ABI calls, every step from pinned host
    # noise: (1) the same step as the device-timed one (ICs + run + P(k)) with the
    # binned P(k) read back to the host; (2) ICs + run with the whole particle
    # state (disp, vel) read back instead
    e2e = e2e_state = None
    if args.e2e_steps > 0:
        nb = WORKLOAD["pk_bins"]

        def timed(call):
            call()
            if ws > 1:
                dist.barrier()
            te = time.perf_counter()
            for _ in range(args.e2e_steps):
                call()
            torch.cuda.synchronize()
            return max_over_ranks(time.perf_counter() - te, ws, dev)

        e2e_s = timed(lambda: pm.simulate_pk_host(noise_host, WORKLOAD["pk_mesh"], nb))
        e2e = {"value": whole_job_rate(N * cfg.n_steps * args.e2e_steps, ws, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": 3 * 8 * nb, "steps": args.e2e_steps,
               "ms_per_step": e2e_s * 1e3 / args.e2e_steps,
               "call": "pm_simulate_pk_host: host noise -> ICs + 6 steps + P(k) -> host P(k)"}
        d_host = torch.empty((1, 3, N), dtype=torch.float32, pin_memory=True)
        v_host = torch.empty((1, 3, N), dtype=torch.float32, pin_memory=True)
        es_s = timed(lambda: pm.simulate_host(noise_host, d_host, v_host))
        e2e_state = {"value": whole_job_rate(N * cfg.n_steps * args.e2e_steps, ws, es_s), "unit": UNIT,
                     "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": 2 * 3 * 4 * N, "steps": args.e2e_steps,
                     "ms_per_step": es_s * 1e3 / args.e2e_steps,
                     "call": "pm_simulate_host: host noise -> ICs + 6 steps -> host disp, vel (no P(k))",
                     "host_link_gbs": host_link_gbs(d_host)}

    # roofline of the dominant kernel (largest share of the timed region)
    alg = algorithmic_bytes(n, cfg.n_mesh, cfg.n_steps)
    peak, peak_kind = measured_peaks()
    kernels = {}
    for name, p in prof.items():
        if p["calls"] == 0:
            continue
        per = p["ms"] / p["calls"]
        entry = {"ms_per_launch": per, "launches": p["calls"], "share": p["ms"] / ms}
        if name in alg:
            entry["gbs"] = alg[name] / (per / 1e3) / 1e9
            entry["frac"] = entry["gbs"] / peak
        kernels[name] = entry
    dom = max((k for k in kernels if k in alg), key=lambda k: kernels[k]["share"])
    traffic = measured_traffic(dom) if (n, cfg.n_mesh) == (512, 512) else None
    roof = {"kernel": dom, "bound": "hbm", "achieved": kernels[dom]["gbs"], "peak": peak, "unit": "GB/s",
            "frac": kernels[dom]["frac"], "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs",
            "algorithmic_bytes_per_launch": alg[dom]}
    launches = sum(p["launches"] for p in prof.values())

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": WORKLOAD, "roofline": roof, "kernels": kernels, "gpu_launches": int(launches),
            "e2e": e2e, "e2e_state": e2e_state,
            "clocks": clock_info,
            "ms_per_pm_step": ms / args.steps / cfg.n_steps}
    if not args.no_extra:
        cmp = cufft_comparison(cfg.n_mesh, dev)
        cmp["ms_own_passes"] = sum(kernels[k]["ms_per_launch"] for k in
                                   ("fft_x_fwd", "fft_y_fwd", "fft_z_green", "fft_y_inv", "fft_x_inv") if k in kernels)
        line["cufft_comparison"] = cmp
        line["adjoint"] = adjoint_benchmark(dev)
        line["scaleup"] = scaleup_benchmark(dev)
        line["deconvolve"] = deconvolve_benchmark(dev)
        line["lpt2_ic"] = lpt2_ic_benchmark(dev)
        line["jvp"] = jvp_benchmark(dev)
        line["nufft"] = nufft_benchmark(dev)
    if not args.no_serving:
        line["serving"] = serving_benchmark(args.serve_requests, dev)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    if rank == 0:
        print(json.dumps(line), flush=True)
    pm.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
