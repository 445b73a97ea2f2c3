"""ctypes declarations of the C ABI in include/pmgb.h (argument marshalling only).

Loading fails loudly when libpmgb.so is missing: there is no fallback path.
"""
import ctypes
import re
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_size_t, c_void_p
from pathlib import Path

PKG = Path(__file__).resolve().parent
HEADER = PKG.parent / "include" / "pmgb.h"
LIB_PATH = PKG / "libpmgb.so"

PM_OK = 0
ERRORS = {-1: "PM_ERR_ARG", -2: "PM_ERR_CUDA", -3: "PM_ERR_OOM", -4: "PM_ERR_STATE", -5: "PM_ERR_UNSUPPORTED"}


class PmConfig(ctypes.Structure):
    _fields_ = [
        ("n_part", c_int32), ("n_mesh", c_int32), ("box", c_double), ("order", c_int32),
        ("interlace", c_int32), ("grad_order", c_int32), ("lap_order", c_int32),
        ("omega_m", c_double), ("h", c_double), ("n_s", c_double), ("sigma8", c_double),
        ("a_ini", c_double), ("a_end", c_double), ("n_steps", c_int32), ("stepper", c_int32),
        ("time_var", c_int32), ("zero_corner", c_int32), ("batch", c_int32), ("pk_mesh_max", c_int32),
        ("deconvolve", c_int32), ("lpt_order", c_int32), ("nufft", c_int32),
    ]


_FP = POINTER(ctypes.c_float)
_SIGS = {
    "pm_config_default": (None, [POINTER(PmConfig)]),
    "pm_workspace_bytes": (c_int32, [POINTER(PmConfig), POINTER(c_size_t)]),
    "pm_init": (c_int32, [POINTER(PmConfig), c_void_p, POINTER(c_void_p)]),
    "pm_destroy": (None, [c_void_p]),
    "pm_last_error": (c_char_p, [c_void_p]),
    "pm_set_stream": (c_int32, [c_void_p, c_void_p]),
    "pm_step_table": (c_int32, [c_void_p, POINTER(c_double), c_int32]),
    "pm_host_step_table": (c_int32, [POINTER(PmConfig), POINTER(c_double), c_int32]),
    "pm_growth": (c_int32, [c_void_p, c_double, POINTER(c_double)]),
    "pm_ic_zeldovich": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pm_ic_zeldovich_slot": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "pm_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32]),
    "pm_run": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32]),
    "pm_set_slots": (c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int32)]),
    "pm_step_slots": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "pm_power_spectrum": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, POINTER(c_double),
                                    POINTER(c_double), POINTER(c_int64)]),
    "pm_density": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p]),
    "pm_force_mesh": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "pm_interp": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "pm_adjoint": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32]),
    "pm_jvp": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32]),
    "pm_power_spectrum_jvp": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, POINTER(c_double),
                                        POINTER(c_double), POINTER(c_double), POINTER(c_int64)]),
    "pm_ic_adjoint": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_double)]),
    "pm_density_vjp": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
    "pm_power_spectrum_async": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p]),
    "pm_power_spectrum_finish": (c_int32, [c_void_p, c_int32, c_int32, POINTER(c_double), POINTER(c_double),
                                           POINTER(c_double), POINTER(c_int64)]),
    "pm_simulate_pk_host": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, POINTER(c_double),
                                      POINTER(c_double), POINTER(c_int64)]),
    "pm_power_spectrum_static": (c_int32, [c_void_p, c_int32, c_double, c_int32, c_int32, c_void_p,
                                           POINTER(c_double), POINTER(c_double), POINTER(c_int64)]),
    "pm_profile": (c_int32, [c_void_p, c_int32]),
    "pm_profile_read": (c_int32, [c_void_p, POINTER(c_double), POINTER(c_int64), POINTER(c_int64), c_int32]),
    "pm_simulate_host": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
}

_lib = None


def header_functions():
    """Names of the functions include/pmgb.h declares."""
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z_0-9]+)\s*\(", text)))


def load(path=None):
    """Load libpmgb.so and declare its signatures (raises if it was not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"{p.name} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(str(p))
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class PmError(RuntimeError):
    pass


def check(rc, handle=None):
    if rc != PM_OK:
        msg = load().pm_last_error(handle)
        raise PmError(f"{ERRORS.get(rc, rc)}: {msg.decode() if msg else ''}")
