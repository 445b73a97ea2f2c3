"""CPU checks of the C ABI: the library builds, loads, exports every function
include/pmgb.h declares, and its host-only entry points (configuration
validation, workspace sizing, the FP64 coefficient table) behave; the
coefficient table (tau1, tau2, alpha, beta per step, Sec. 2.4) matches the oracle."""
import ctypes

import numpy as np
import pytest

from oracle import cosmology
from paper_2510_05206_gb300 import _lib, build
from paper_2510_05206_gb300.pm import Config


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    names = _lib.header_functions()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name
    # and the binding declares them all
    assert set(names) == set(_lib._SIGS), set(names) ^ set(_lib._SIGS)


def test_config_default_matches_table4(lib):
    c = _lib.PmConfig()
    lib.pm_config_default(ctypes.byref(c))
    assert (c.order, c.grad_order, c.lap_order, c.stepper, c.time_var, c.zero_corner) == (2, 4, 0, 0, 0, 1)
    assert c.batch == 1 and c.deconvolve == 0


@pytest.mark.parametrize("field,value", [("n_part", 48), ("n_mesh", 2048), ("order", 5), ("grad_order", 3),
                                         ("batch", 0), ("a_end", 0.01), ("box", -1.0), ("n_steps", 0),
                                         ("deconvolve", 2)])
def test_invalid_config_rejected(lib, field, value):
    c = Config(n_part=32, n_mesh=32)
    setattr(c, field, value)
    out = ctypes.c_size_t()
    cc = c.to_c()
    rc = lib.pm_workspace_bytes(ctypes.byref(cc), ctypes.byref(out))
    assert rc == -1
    assert lib.pm_last_error(None)


@pytest.mark.parametrize("kw", [dict(lpt_order=3), dict(interlace=2), dict(stepper=2), dict(time_var=2),
                                dict(lap_order=5), dict(omega_m=1.5), dict(sigma8=0.0), dict(a_ini=1e-5),
                                dict(a_end=4.0), dict(pk_mesh_max=48), dict(nufft=2),
                                dict(nufft=1, grad_order=4), dict(nufft=1, grad_order=0, interlace=1),
                                dict(nufft=1, grad_order=0, deconvolve=1),
                                dict(nufft=1, grad_order=0, n_mesh=1024),
                                dict(n_part=1024, n_mesh=1024, batch=2)])
def test_invalid_option_combinations_rejected(lib, kw):
    c = Config(n_part=32, n_mesh=32)
    for k, v in kw.items():
        setattr(c, k, v)
    out = ctypes.c_size_t()
    cc = c.to_c()
    assert lib.pm_workspace_bytes(ctypes.byref(cc), ctypes.byref(out)) == -1
    assert lib.pm_last_error(None)


def test_valid_option_combinations_size_their_workspace(lib):
    def ws(**kw):
        c = Config(**kw).to_c()
        out = ctypes.c_size_t()
        assert lib.pm_workspace_bytes(ctypes.byref(c), ctypes.byref(out)) == 0, lib.pm_last_error(None)
        return out.value
    base = ws(n_part=64, n_mesh=64)
    # the NUFFT grid is twice the mesh per dimension: 8x the mesh workspace
    assert ws(n_part=64, n_mesh=64, nufft=1, grad_order=0) > 4 * base
    # an interlaced second grid doubles the meshes
    assert ws(n_part=64, n_mesh=64, interlace=1) > 1.5 * base
    for kw in (dict(order=4, deconvolve=1), dict(lpt_order=2), dict(stepper=1, time_var=1),
               dict(grad_order=6, lap_order=4), dict(pk_mesh_max=128)):
        assert ws(n_part=64, n_mesh=64, **kw) >= base


def test_workspace_bytes_scales_with_batch(lib):
    def ws(**kw):
        c = Config(**kw).to_c()
        out = ctypes.c_size_t()
        assert lib.pm_workspace_bytes(ctypes.byref(c), ctypes.byref(out)) == 0
        return out.value
    b1 = ws(n_part=128, n_mesh=128, batch=1)
    b4 = ws(n_part=128, n_mesh=128, batch=4)
    assert 3.5 * b1 < b4 < 4.1 * b1
    # 512^3: density + 3 padded spectra + 3 force meshes ~ 3.7 GB
    assert 3.0e9 < ws(n_part=512, n_mesh=512) < 4.5e9


@pytest.mark.parametrize("stepper,time_var,om", [(0, 0, 0.3), (0, 1, 0.3), (1, 0, 0.3), (0, 0, 0.3158)])
def test_host_step_table_matches_oracle(lib, stepper, time_var, om):
    c = Config(n_part=32, n_mesh=32, n_steps=10, omega_m=om, stepper=stepper, time_var=time_var).to_c()
    out = np.zeros((10, 7))
    rc = lib.pm_host_step_table(ctypes.byref(c), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 10)
    assert rc == 0
    g = cosmology.Growth(om)
    ref = cosmology.step_table(g, 0.02, 1.0, 10, ["bullfrog", "fastpm"][stepper], ["D", "a"][time_var])
    np.testing.assert_allclose(out, ref, rtol=1e-9, atol=1e-12)


def test_float32_bin_rule_equals_fp64_for_every_mesh_mode():
    # The P(k) z pass takes each mode's bin as floor(sqrt(|m|^2) - 1/2) in float32
    # (correctly rounded square root); the oracle bins |k| / k_F in FP64.  Every
    # integer |m|^2 that a mesh of up to 1024^3 cells reaches (<= 3 * 512^2) gets the
    # same bin in both precisions: no |m| lies close enough to a bin edge.
    s = np.arange(0, 3 * 512 * 512 + 1)
    b32 = np.floor(np.sqrt(s.astype(np.float32)) - np.float32(0.5)).astype(np.int64)
    b64 = np.floor(np.sqrt(s.astype(np.float64)) - 0.5).astype(np.int64)
    np.testing.assert_array_equal(b32, b64)


def test_missing_library_fails_loudly(tmp_path):
    # the product path has no CPU fallback: without the built library, loading raises
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load(tmp_path / "libpmgb.so")


@pytest.mark.parametrize("name", ["pm_set_stream", "pm_step_table", "pm_growth", "pm_ic_zeldovich",
                                  "pm_ic_zeldovich_slot", "pm_step", "pm_run", "pm_set_slots", "pm_step_slots",
                                  "pm_power_spectrum", "pm_power_spectrum_async", "pm_power_spectrum_finish",
                                  "pm_power_spectrum_jvp", "pm_density", "pm_force_mesh", "pm_interp",
                                  "pm_adjoint", "pm_jvp", "pm_ic_adjoint", "pm_density_vjp", "pm_profile",
                                  "pm_profile_read", "pm_simulate_host", "pm_simulate_pk_host"])
def test_null_handle_is_an_argument_error(lib, name):
    # every call that takes a handle rejects NULL with PM_ERR_ARG before any CUDA work
    fn = getattr(lib, name)
    scalar = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t)
    args = [0 if t in scalar else None for t in fn.argtypes]
    args[0] = None
    assert fn(*args) == -1
