"""GPU parity: every stage of the PM hot path through the C ABI against the FP64
oracle on the same seeded inputs (Sec. 2.2 ICs, Sec. 2.4 Eq. dkd, Sec. 2.5
deposit / Poisson force / interpolation, Sec. 2.9 P(k)).

Tolerances (float32 path vs float64 oracle):
* meshes and per-particle fields: max |gpu - oracle| <= 2e-5 * max |oracle|
  (float32 rounding ~6e-8 per operation; an FFT of n points adds ~log2 n
  rounding steps, the deposit sums <= 27 weights per cell);
* full runs: max_i |Psi_gpu - Psi_oracle| <= 1e-4 * rms |Psi_oracle| and each
  P(k) bin within 1e-4 relative (the required parity).
"""
import math

import numpy as np
import pytest
import torch

from oracle import cosmology, mesh, nbody
from paper_2510_05206_gb300 import PM, Config, inputs

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


def _np(t):
    return t.double().cpu().numpy()


def _rel_max(got, ref):
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


@pytest.mark.parametrize("n_part,n_mesh,order", [(32, 32, 2), (32, 64, 2), (32, 32, 3), (64, 32, 3), (16, 64, 2),
                                                 (32, 32, 4), (32, 64, 4)])
def test_density_deposit(n_part, n_mesh, order):
    L = 100.0
    pm = PM(Config(n_part=n_part, n_mesh=n_mesh, box=L, order=order), device=DEV)
    Psi = inputs.random_displacements(n_part, scale=3.0 * L / n_mesh, seed=1)
    delta = _np(pm.density(_t(Psi[None]), n_mesh, order))[0]
    X = np.mod(nbody.lattice(n_part, L) + Psi, L)
    ref = mesh.density_contrast(X, n_mesh, L, order)
    assert _rel_max(delta, ref) < 2e-5
    # mass conservation: sum delta = 0 to float32 rounding
    assert abs(delta.sum()) < 1e-4 * n_mesh ** 3 ** 0.5 + 1e-3


@pytest.mark.parametrize("n_part,n_mesh,order", [(32, 32, 2), (64, 64, 2), (32, 32, 3), (32, 64, 2), (32, 64, 3), (32, 32, 4), (32, 64, 4)])
def test_density_deposit_structured(n_part, n_mesh, order):
    # tile-window paths of the deposit: jittered columns, collapsed columns (many
    # particles per cell) and particles far outside their tile's window
    L = 100.0
    pm = PM(Config(n_part=n_part, n_mesh=n_mesh, box=L, order=order), device=DEV)
    Psi = inputs.structured_displacements(n_part, L / n_mesh, seed=11)
    delta = _np(pm.density(_t(Psi[None]), n_mesh, order))[0]
    X = np.mod(nbody.lattice(n_part, L) + Psi, L)
    ref = mesh.density_contrast(X, n_mesh, L, order)
    assert _rel_max(delta, ref) < 2e-5
    assert abs(delta.sum()) < 1e-4 * n_mesh ** 3 ** 0.5 + 1e-3


@pytest.mark.parametrize("n,order,pre", [(32, 2, 0), (64, 2, 0), (32, 2, 1), (32, 3, 0)])
def test_kick_drift_structured(n, order, pre):
    # one DKD step from structured positions through the column-walk interpolation
    # (CIC, mesh = lattice: tap planes reused for columns in the same or next cell)
    # against the oracle step; pre = 1 carries pre-drifted positions (a 2-step run)
    L = 64.0
    kw = dict(n_part=n, n_mesh=n, box=L, order=order, n_steps=2)
    pm = PM(Config(**kw), device=DEV)
    Psi = inputs.structured_displacements(n, L / n, seed=12)
    V = inputs.random_displacements(n, scale=0.3, seed=13)
    d, v = _t(Psi[None]), _t(V[None])
    ocfg = nbody.Config(**kw)
    tab = cosmology.step_table(ocfg.get_growth(), ocfg.a_ini, ocfg.a_end, 2)
    P1, V1 = nbody.step(ocfg, Psi, V, tab[0], nbody.lattice(n, L))
    if pre:
        pm.run(d, v, 0, 2)
        P1, V1 = nbody.step(ocfg, P1, V1, tab[1], nbody.lattice(n, L))
    else:
        pm.step(d, v, 0)
    assert _disp_err(_np(d)[0], P1) < 1e-4
    assert _disp_err(_np(v)[0], V1) < 1e-4


@pytest.mark.parametrize("n,grad,lap,order,dec", [(32, 4, 0, 2, 0), (64, 4, 0, 2, 0), (32, 0, 0, 2, 0),
                                                   (32, 2, 2, 2, 0), (16, 6, 4, 2, 0), (128, 4, 0, 2, 0),
                                                   (32, 4, 0, 2, 1), (32, 0, 0, 3, 1), (64, 6, 2, 3, 1)])
def test_force_mesh(n, grad, lap, order, dec):
    # dec = 1: the density spectrum is divided by the squared order-p kernel (Table 1)
    L = 300.0
    pm = PM(Config(n_part=n, n_mesh=n, box=L, grad_order=grad, lap_order=lap, order=order, deconvolve=dec),
            device=DEV)
    d = inputs.random_field(n, seed=2)
    g = _np(pm.force_mesh(_t(d[None])))[0]
    ref = mesh.force_field(d, L, grad, lap, deconvolve_order=order if dec else 0)
    for c in range(3):
        assert _rel_max(g[c], ref[c]) < 2e-5, c


@pytest.mark.parametrize("n_part,n_mesh,order", [(32, 32, 2), (32, 64, 3), (64, 32, 2), (32, 32, 4)])
def test_interp(n_part, n_mesh, order):
    L = 80.0
    pm = PM(Config(n_part=n_part, n_mesh=n_mesh, box=L, order=order), device=DEV)
    g = np.stack([inputs.random_field(n_mesh, seed=10 + c) for c in range(3)])
    Psi = inputs.random_displacements(n_part, scale=4.0 * L / n_mesh, seed=3)
    acc = _np(pm.interp(_t(Psi[None]), _t(g[None])))[0]
    X = np.mod(nbody.lattice(n_part, L) + Psi, L)
    for c in range(3):
        ref = mesh.gather(g[c], X, L, order)
        assert _rel_max(acc[c], ref) < 2e-5


@pytest.mark.parametrize("n,corner", [(32, 1), (64, 1), (32, 0)])
def test_zeldovich_ic(n, corner):
    L = 256.0
    cfg = Config(n_part=n, n_mesh=n, box=L, zero_corner=corner)
    pm = PM(cfg, device=DEV)
    w = inputs.white_noise(n, seed=4)
    disp, vel = pm.ic_zeldovich(_t(w.reshape(1, -1)))
    ocfg = nbody.Config(n_part=n, n_mesh=n, box=L, zero_corner=bool(corner))
    P0, V0 = nbody.zeldovich_ic(ocfg, w)
    assert _rel_max(_np(vel)[0], V0) < 2e-5
    assert _rel_max(_np(disp)[0], P0) < 2e-5


@pytest.mark.parametrize("n", [32, 64])
def test_lpt2_ic(n):
    # 2LPT ICs against the oracle; the second-order part alone (2LPT minus Zel'dovich
    # velocities = 2 D psi2) at a_ini = 0.1, where it is large enough to be resolved
    # by the float32 difference
    L = 256.0
    kw = dict(n_part=n, n_mesh=n, box=L, a_ini=0.1)
    w = inputs.white_noise(n, seed=4)
    d1, v1 = PM(Config(**kw), device=DEV).ic_zeldovich(_t(w.reshape(1, -1)))
    d2, v2 = PM(Config(lpt_order=2, **kw), device=DEV).ic_zeldovich(_t(w.reshape(1, -1)))
    P1, V1 = nbody.zeldovich_ic(nbody.Config(**kw), w)
    P2, V2 = nbody.zeldovich_ic(nbody.Config(lpt_order=2, **kw), w)
    assert _rel_max(_np(d2)[0], P2) < 2e-5
    assert _rel_max(_np(v2)[0], V2) < 2e-5
    assert _rel_max(_np(v2)[0] - _np(v1)[0], V2 - V1) < 2e-3
    assert _rel_max(_np(d2)[0] - _np(d1)[0], P2 - P1) < 2e-3


def _run_pair(cfg_kw, seed, n_bins=None):
    cfg = Config(**cfg_kw)
    pm = PM(cfg, device=DEV)
    w = inputs.white_noise(cfg.n_part, seed=seed)
    disp, vel = pm.ic_zeldovich(_t(w.reshape(1, -1)))
    pm.run(disp, vel)
    okw = dict(n_part=cfg.n_part, n_mesh=cfg.n_mesh, box=cfg.box, order=cfg.order,
               interlace=bool(cfg.interlace), grad_order=cfg.grad_order, lap_order=cfg.lap_order,
               n_steps=cfg.n_steps, a_ini=cfg.a_ini, a_end=cfg.a_end,
               stepper=["bullfrog", "fastpm"][cfg.stepper], time_var=["D", "a"][cfg.time_var],
               deconvolve=bool(cfg.deconvolve), lpt_order=max(cfg.lpt_order, 1))
    ocfg = nbody.Config(**okw)
    P0, V0 = nbody.zeldovich_ic(ocfg, w)
    P1, V1 = nbody.run(ocfg, P0, V0)
    return pm, disp, vel, P1, V1


def _disp_err(got, ref):
    return np.max(np.abs(got - ref)) / np.sqrt(np.mean(np.sum(ref ** 2, axis=0)))


def test_full_run_config1_parity():
    # 32^3 particles on a 32^3 mesh, L = 256 Mpc/h, CIC, 6 BullFrog steps a = 0.02 -> 1
    pm, disp, vel, P1, V1 = _run_pair(dict(n_part=32, n_mesh=32, box=256.0, n_steps=6), seed=1)
    d = _np(disp)[0]
    v = _np(vel)[0]
    assert _disp_err(d, P1) < 1e-4
    assert _disp_err(v, V1) < 1e-4
    # final power spectrum, 16 bins, per-bin relative error
    k, pk, cnt = pm.power_spectrum(disp, 32, 16)
    X = np.mod(nbody.lattice(32, 256.0) + P1, 256.0)
    kr, pr, cr = mesh.power_spectrum(mesh.density_contrast(X, 32, 256.0, 2), 256.0, 16)
    np.testing.assert_array_equal(cnt[0], cr)
    np.testing.assert_allclose(k[0], kr, rtol=1e-12)
    assert np.max(np.abs(pk[0] / pr - 1)) < 1e-4


@pytest.mark.parametrize("kw", [
    dict(n_part=32, n_mesh=64, box=125.0, order=3, interlace=1, n_steps=10),      # config-2 settings, reduced
    dict(n_part=32, n_mesh=32, box=200.0, order=3, n_steps=4, stepper=1),         # FastPM
    dict(n_part=16, n_mesh=32, box=100.0, order=2, n_steps=5, time_var=1, grad_order=2, lap_order=2),
    dict(n_part=32, n_mesh=32, box=256.0, order=2, n_steps=3, grad_order=0),                # exact i k gradient
    dict(n_part=32, n_mesh=64, box=200.0, order=2, n_steps=3, grad_order=6, lap_order=4),
    dict(n_part=32, n_mesh=32, box=150.0, order=2, interlace=1, n_steps=3, grad_order=0),   # 6 inverse FFTs
    dict(n_part=32, n_mesh=32, box=256.0, order=2, n_steps=6, deconvolve=1),                 # option (ii): N_g = N + deconv.
    dict(n_part=32, n_mesh=32, box=200.0, order=3, n_steps=4, deconvolve=1, interlace=1),
    dict(n_part=32, n_mesh=32, box=256.0, order=2, n_steps=6, lpt_order=2),                 # 2LPT ICs
    dict(n_part=32, n_mesh=32, box=256.0, order=4, n_steps=4, deconvolve=1),                 # PCS + deconvolution
    dict(n_part=32, n_mesh=64, box=200.0, order=4, n_steps=3, interlace=1),                  # PCS, interlaced
    dict(n_part=64, n_mesh=32, box=256.0, order=2, n_steps=4, lpt_order=2),                 # mesh smaller than lattice
])
def test_full_run_variants_parity(kw):
    pm, disp, vel, P1, V1 = _run_pair(kw, seed=2)
    assert _disp_err(_np(disp)[0], P1) < 1e-4
    assert _disp_err(_np(vel)[0], V1) < 1e-4


def test_power_spectrum_stage():
    n, L = 64, 500.0
    pm = PM(Config(n_part=32, n_mesh=32, box=L, pk_mesh_max=64), device=DEV)
    Psi = inputs.random_displacements(32, scale=6.0, seed=5)
    k, pk, cnt = pm.power_spectrum(_t(Psi[None]), n, 32)
    X = np.mod(nbody.lattice(32, L) + Psi, L)
    kr, pr, cr = mesh.power_spectrum(mesh.density_contrast(X, n, L, 2), L, 32)
    np.testing.assert_array_equal(cnt[0], cr)
    ok = cr > 0
    assert np.max(np.abs(pk[0][ok] / pr[ok] - 1)) < 1e-4


def test_power_spectrum_on_smaller_mesh_than_handle():
    # P(k) meshes below n_mesh use their own twiddle tables (regression test)
    n_part, L = 64, 300.0
    pm = PM(Config(n_part=n_part, n_mesh=64, box=L), device=DEV)
    Psi = inputs.random_displacements(n_part, scale=5.0, seed=6)
    X = np.mod(nbody.lattice(n_part, L) + Psi, L)
    for n, nb in ((32, 12), (16, 8), (64, 32)):
        k, pk, cnt = pm.power_spectrum(_t(Psi[None]), n, nb)
        kr, pr, cr = mesh.power_spectrum(mesh.density_contrast(X, n, L, 2), L, nb)
        np.testing.assert_array_equal(cnt[0], cr)
        assert np.max(np.abs(pk[0] / pr - 1)) < 1e-4


def test_batched_slots_match_single_runs():
    n, L = 32, 256.0
    B = 3
    w = inputs.white_noise(n, seed=7, batch=B)
    pmb = PM(Config(n_part=n, n_mesh=n, box=L, batch=B), device=DEV)
    disp, vel = pmb.ic_zeldovich(_t(w.reshape(B, -1)))
    pmb.run(disp, vel)
    pm1 = PM(Config(n_part=n, n_mesh=n, box=L), device=DEV)
    for b in range(B):
        d1, v1 = pm1.ic_zeldovich(_t(w[b].reshape(1, -1)))
        pm1.run(d1, v1)
        # identical kernels and data: equal up to the order of float atomics in the deposit
        assert _disp_err(_np(disp)[b], _np(d1)[0]) < 1e-5


def test_slot_schedule_mixed_steps():
    # continuous batching: slots at different step indices of different-length
    # runs in one launch give the same states as separate runs
    n, L = 32, 256.0
    pm = PM(Config(n_part=n, n_mesh=n, box=L, batch=2), device=DEV)
    w = inputs.white_noise(n, seed=8, batch=2)
    disp, vel = pm.ic_zeldovich(_t(w.reshape(2, -1)))
    nsteps = [4, 6]
    for s in range(6):
        step = [s if s < nsteps[0] else -1, s]
        pm.set_slots(nsteps, step)
        pm.step_slots(disp, vel)
    for b, ns in enumerate(nsteps):
        pmb = PM(Config(n_part=n, n_mesh=n, box=L, n_steps=ns), device=DEV)
        d1, v1 = pmb.ic_zeldovich(_t(w[b].reshape(1, -1)))
        pmb.run(d1, v1)
        assert _disp_err(_np(disp)[b], _np(d1)[0]) < 1e-5


@pytest.mark.parametrize("n_steps", [1, 2])
def test_shortest_runs_parity(n_steps):
    # one step (no carried pre-drift) and two steps (the shortest run that carries it)
    pm, disp, vel, P1, V1 = _run_pair(dict(n_part=32, n_mesh=32, box=256.0, n_steps=n_steps), seed=11)
    assert _disp_err(_np(disp)[0], P1) < 1e-4
    assert _disp_err(_np(vel)[0], V1) < 1e-4


@pytest.mark.parametrize("cuts", [(3,), (1, 2, 5), (1, 2, 3, 4, 5)])
def test_run_in_segments_equals_one_run(cuts):
    # a run split into step ranges leaves the same state as one call: each call
    # starts and ends on plain positions, whatever it carries between its steps
    n, L = 32, 256.0
    w = _t(inputs.white_noise(n, seed=12).reshape(1, -1))
    pm = PM(Config(n_part=n, n_mesh=n, box=L), device=DEV)
    d0, v0 = pm.ic_zeldovich(w)
    pm.run(d0, v0)
    d1, v1 = pm.ic_zeldovich(w)
    edges = (0,) + cuts + (6,)
    for b, e in zip(edges[:-1], edges[1:]):
        pm.run(d1, v1, b, e)
    # the split only regroups float additions of the drifts (X + t2 V + t1' V)
    assert _disp_err(_np(d1)[0], _np(d0)[0]) < 1e-5
    assert _disp_err(_np(v1)[0], _np(v0)[0]) < 1e-5


def test_empty_step_range_is_a_no_op():
    n = 16
    pm = PM(Config(n_part=n, n_mesh=n, box=100.0), device=DEV)
    d, v = pm.ic_zeldovich(_t(inputs.white_noise(n, seed=13).reshape(1, -1)))
    d_ref, v_ref = d.clone(), v.clone()
    pm.run(d, v, 3, 3)
    torch.cuda.synchronize()
    assert torch.equal(d, d_ref) and torch.equal(v, v_ref)


def test_simulate_host_matches_device_path():
    n, L = 32, 256.0
    pm = PM(Config(n_part=n, n_mesh=n, box=L), device=DEV)
    w = inputs.white_noise(n, seed=9).reshape(1, -1).astype(np.float32)
    dh, vh = pm.simulate_host(torch.from_numpy(w).pin_memory())
    d, v = pm.ic_zeldovich(_t(w))
    pm.run(d, v)
    assert _disp_err(dh[0].double().numpy(), _np(d)[0]) < 1e-5


def test_simulate_pk_host_matches_device_path():
    # the whole analysis step from host noise to host P(k) equals ICs + run + P(k)
    # on device buffers (same kernels, same inputs)
    n, L = 32, 256.0
    pm = PM(Config(n_part=n, n_mesh=n, box=L), device=DEV)
    w = inputs.white_noise(n, seed=10).reshape(1, -1).astype(np.float32)
    kh, pkh, ch = pm.simulate_pk_host(torch.from_numpy(w).pin_memory(), 32, 16)
    d, v = pm.ic_zeldovich(_t(w))
    pm.run(d, v)
    k, pk, c = pm.power_spectrum(d, 32, 16)
    np.testing.assert_array_equal(ch, c)
    np.testing.assert_array_equal(kh, k)
    assert np.max(np.abs(pkh / pk - 1)) < 1e-5
    with pytest.raises(ValueError):
        pm.simulate_pk_host(_t(w))          # device tensor: not a host buffer


def test_power_spectrum_async_matches_sync():
    # enqueue for two states back to back, finish both after one synchronisation
    n, L = 32, 256.0
    pm = PM(Config(n_part=n, n_mesh=n, box=L), device=DEV)
    w = inputs.white_noise(n, seed=14).reshape(1, -1)
    d0, v0 = pm.ic_zeldovich(_t(w))
    d1, v1 = d0.clone(), v0.clone()
    pm.run(d1, v1)
    sums = torch.empty((2, 1, 16), dtype=torch.float64, device=DEV)
    pm.power_spectrum_async(d0, sums[0], 32, 16)
    pm.power_spectrum_async(d1, sums[1], 32, 16)
    torch.cuda.synchronize()
    for i, d in enumerate((d0, d1)):
        ka, pka, ca = pm.power_spectrum_finish(sums[i], 32, 16)
        k, pk, c = pm.power_spectrum(d, 32, 16)
        np.testing.assert_array_equal(ca, c)
        np.testing.assert_array_equal(ka, k)
        assert np.max(np.abs(pka / pk - 1)) < 1e-12


def test_step_table_matches_oracle():
    pm = PM(Config(n_part=16, n_mesh=16, box=100.0, n_steps=7), device=DEV)
    ref = cosmology.step_table(cosmology.Growth(0.3), 0.02, 1.0, 7)
    np.testing.assert_allclose(pm.step_table(), ref, rtol=1e-9, atol=1e-12)


def test_invalid_calls_raise():
    pm = PM(Config(n_part=16, n_mesh=16, box=100.0), device=DEV)
    d, v = pm.new_state()
    with pytest.raises(RuntimeError):
        pm.step(d, v, 99)
    with pytest.raises(RuntimeError):
        pm.power_spectrum(d, 2048, 8)


@pytest.mark.parametrize("n_part,n_mesh", [(16, 16), (32, 16), (16, 32)])
def test_nufft_run_parity(n_part, n_mesh):
    # NUFFT force (ES kernel, width 5, grid 2 n_mesh, n_mesh band) against the
    # oracle's FP64 NUFFT (itself within ~1e-4 of the exact band-limited DFT)
    kw = dict(n_part=n_part, n_mesh=n_mesh, box=64.0, n_steps=3, grad_order=0)
    pm = PM(Config(nufft=1, **kw), device=DEV)
    w = inputs.white_noise(n_part, seed=51)
    d, v = pm.ic_zeldovich(_t(w.reshape(1, -1)))
    pm.run(d, v)
    ocfg = nbody.Config(nufft=True, **kw)
    P0, V0 = nbody.zeldovich_ic(ocfg, w)
    P1, V1 = nbody.run(ocfg, P0, V0)
    assert _disp_err(_np(d)[0], P1) < 1e-4
    assert _disp_err(_np(v)[0], V1) < 1e-4


def test_nufft_rejects_unsupported_calls():
    pm = PM(Config(n_part=16, n_mesh=16, box=64.0, grad_order=0, nufft=1), device=DEV)
    d, v = pm.new_state()
    with pytest.raises(RuntimeError):
        pm.adjoint(d, v, torch.zeros_like(d), torch.zeros_like(v))
    with pytest.raises(RuntimeError):
        PM(Config(n_part=16, n_mesh=16, box=64.0, grad_order=4, nufft=1), device=DEV)
