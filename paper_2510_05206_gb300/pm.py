"""Thin torch binding of libpmgb (include/pmgb.h): same names, argument
marshalling only.  Every step of the PM path runs in the library's CUDA
kernels; tensors only supply device memory and the current stream."""
import ctypes
from dataclasses import dataclass, fields

import numpy as np
import torch

from . import _lib


@dataclass
class Config:
    n_part: int = 64
    n_mesh: int = 64
    box: float = 256.0
    order: int = 2
    interlace: int = 0
    grad_order: int = 4
    lap_order: int = 0
    omega_m: float = 0.3
    h: float = 0.7
    n_s: float = 0.96
    sigma8: float = 0.8
    a_ini: float = 0.02
    a_end: float = 1.0
    n_steps: int = 6
    stepper: int = 0
    time_var: int = 0
    zero_corner: int = 1
    batch: int = 1
    pk_mesh_max: int = 0
    deconvolve: int = 0         # divide the force density by the squared kernel (Table 1 W^)
    lpt_order: int = 1          # initial conditions: 1 = Zel'dovich, 2 = 2LPT
    nufft: int = 0              # force by the NUFFT (ES kernel on a 2 n_mesh grid, n_mesh band)

    def to_c(self):
        c = _lib.PmConfig()
        for f in fields(self):
            setattr(c, f.name, getattr(self, f.name))
        return c


def workspace_bytes(cfg: Config) -> int:
    lib = _lib.load()
    out = ctypes.c_size_t()
    c = cfg.to_c()
    _lib.check(lib.pm_workspace_bytes(ctypes.byref(c), ctypes.byref(out)))
    return out.value


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class PM:
    """One libpmgb handle serving ``cfg.batch`` simulations of the same size."""

    def __init__(self, cfg: Config, device="cuda"):
        self.lib = _lib.load()
        self.cfg = cfg
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("libpmgb runs on CUDA devices only")
        torch.cuda.init()
        with torch.cuda.device(self.device):
            h = ctypes.c_void_p()
            c = cfg.to_c()
            stream = torch.cuda.current_stream(self.device).cuda_stream
            _lib.check(self.lib.pm_init(ctypes.byref(c), ctypes.c_void_p(stream), ctypes.byref(h)))
        self.h = h
        self.N = cfg.n_part ** 3
        self.B = cfg.batch

    def close(self):
        if getattr(self, "h", None):
            self.lib.pm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    def _stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        _lib.check(self.lib.pm_set_stream(self.h, ctypes.c_void_p(s)), self.h)

    def _check(self, rc):
        _lib.check(rc, self.h)

    def _state_ok(self, t, name, shape):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
        if t.numel() != int(np.prod(shape)):
            raise ValueError(f"{name} has {t.numel()} elements, expected {shape}")

    def new_state(self):
        shape = (self.B, 3, self.N)
        return (torch.zeros(shape, device=self.device, dtype=torch.float32),
                torch.zeros(shape, device=self.device, dtype=torch.float32))

    # ------------------------------------------------------------ API
    def step_table(self):
        out = np.zeros((self.cfg.n_steps, 7))
        self._check(self.lib.pm_step_table(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           self.cfg.n_steps))
        return out

    def growth(self, a):
        out = np.zeros(3)
        self._check(self.lib.pm_growth(self.h, float(a), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def ic_zeldovich(self, noise, disp=None, vel=None):
        self._state_ok(noise, "noise", (self.B, self.N))
        if disp is None:
            disp, vel = self.new_state()
        self._state_ok(disp, "disp", (self.B, 3, self.N))
        self._state_ok(vel, "vel", (self.B, 3, self.N))
        self._stream()
        self._check(self.lib.pm_ic_zeldovich(self.h, _ptr(noise), _ptr(disp), _ptr(vel)))
        return disp, vel

    def ic_zeldovich_slot(self, slot, noise, disp, vel):
        self._stream()
        self._check(self.lib.pm_ic_zeldovich_slot(self.h, int(slot), _ptr(noise), _ptr(disp), _ptr(vel)))

    def step(self, disp, vel, step):
        self._stream()
        self._check(self.lib.pm_step(self.h, _ptr(disp), _ptr(vel), int(step)))

    def run(self, disp, vel, begin=0, end=None):
        self._state_ok(disp, "disp", (self.B, 3, self.N))
        self._state_ok(vel, "vel", (self.B, 3, self.N))
        self._stream()
        end = self.cfg.n_steps if end is None else end
        self._check(self.lib.pm_run(self.h, _ptr(disp), _ptr(vel), int(begin), int(end)))
        return disp, vel

    def set_slots(self, n_steps, step):
        ns = np.ascontiguousarray(n_steps, dtype=np.int32)
        st = np.ascontiguousarray(step, dtype=np.int32)
        if ns.size != self.B or st.size != self.B:
            raise ValueError("one entry per slot expected")
        self._stream()
        self._check(self.lib.pm_set_slots(self.h, ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                          st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))

    def step_slots(self, disp, vel):
        self._stream()
        self._check(self.lib.pm_step_slots(self.h, _ptr(disp), _ptr(vel)))

    def power_spectrum(self, disp, n_mesh=None, n_bins=None):
        n = n_mesh or (self.cfg.pk_mesh_max or self.cfg.n_mesh)
        nb = n_bins or n // 2
        k = np.zeros((self.B, nb))
        pk = np.zeros((self.B, nb))
        cnt = np.zeros((self.B, nb), dtype=np.int64)
        self._stream()
        self._check(self.lib.pm_power_spectrum(
            self.h, _ptr(disp), int(n), int(nb), k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            pk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return k, pk, cnt

    def power_spectrum_async(self, disp, bin_sums, n_mesh=None, n_bins=None):
        """Enqueue P(k) without synchronising: bin_sums, a float64 CUDA tensor of
        B x n_bins values, receives the raw per-bin sums (see power_spectrum_finish)."""
        n = n_mesh or (self.cfg.pk_mesh_max or self.cfg.n_mesh)
        nb = n_bins or n // 2
        if not (bin_sums.is_cuda and bin_sums.dtype == torch.float64 and bin_sums.is_contiguous()
                and bin_sums.numel() == self.B * nb):
            raise ValueError(f"bin_sums must be a contiguous float64 CUDA tensor of {self.B} x {nb} values")
        self._stream()
        self._check(self.lib.pm_power_spectrum_async(self.h, _ptr(disp), int(n), int(nb), _ptr(bin_sums)))

    def power_spectrum_finish(self, bin_sums, n_mesh=None, n_bins=None):
        """(k, P, counts) from the per-bin sums of power_spectrum_async (host copy or
        CUDA tensor; a CUDA tensor is copied to the host, which waits for it)."""
        n = n_mesh or (self.cfg.pk_mesh_max or self.cfg.n_mesh)
        nb = n_bins or n // 2
        sums = np.ascontiguousarray(bin_sums.cpu().numpy() if torch.is_tensor(bin_sums) else bin_sums,
                                    dtype=np.float64)
        k, pk = np.zeros((self.B, nb)), np.zeros((self.B, nb))
        cnt = np.zeros((self.B, nb), dtype=np.int64)
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._check(self.lib.pm_power_spectrum_finish(self.h, int(n), int(nb), dptr(sums), dptr(k), dptr(pk),
                                                      cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return k, pk, cnt

    def density(self, disp, n_mesh=None, order=None):
        n = n_mesh or self.cfg.n_mesh
        out = torch.empty((self.B, n, n, n), device=self.device, dtype=torch.float32)
        self._stream()
        self._check(self.lib.pm_density(self.h, _ptr(disp), int(n), int(order or self.cfg.order), _ptr(out)))
        return out

    def force_mesh(self, delta):
        n = self.cfg.n_mesh
        self._state_ok(delta, "delta", (self.B, n, n, n))
        out = torch.empty((self.B, 3, n, n, n), device=self.device, dtype=torch.float32)
        self._stream()
        self._check(self.lib.pm_force_mesh(self.h, _ptr(delta), _ptr(out)))
        return out

    def interp(self, disp, force):
        out = torch.empty((self.B, 3, self.N), device=self.device, dtype=torch.float32)
        self._stream()
        self._check(self.lib.pm_interp(self.h, _ptr(disp), _ptr(force), _ptr(out)))
        return out

    def adjoint(self, disp, vel, adj_disp, adj_vel, step_end=None):
        """Backward DKD in place: (disp, vel) -> initial state, (adj_disp, adj_vel) -> initial cotangents."""
        for t, nm in ((disp, "disp"), (vel, "vel"), (adj_disp, "adj_disp"), (adj_vel, "adj_vel")):
            self._state_ok(t, nm, (self.B, 3, self.N))
        self._stream()
        end = self.cfg.n_steps if step_end is None else step_end
        self._check(self.lib.pm_adjoint(self.h, _ptr(disp), _ptr(vel), _ptr(adj_disp), _ptr(adj_vel), int(end)))

    def jvp(self, disp, vel, tdisp, tvel, begin=0, end=None):
        """Forward mode in place: advances (disp, vel) and the tangent (tdisp, tvel)
        through steps [begin, end) (default: all)."""
        for t, nm in ((disp, "disp"), (vel, "vel"), (tdisp, "tdisp"), (tvel, "tvel")):
            self._state_ok(t, nm, (self.B, 3, self.N))
        self._stream()
        end = self.cfg.n_steps if end is None else end
        self._check(self.lib.pm_jvp(self.h, _ptr(disp), _ptr(vel), _ptr(tdisp), _ptr(tvel), int(begin), int(end)))

    def power_spectrum_jvp(self, disp, tdisp, n_mesh=None, n_bins=None):
        """(k, P, dP, counts): P(k) of disp and its tangent along tdisp."""
        n = n_mesh or (self.cfg.pk_mesh_max or self.cfg.n_mesh)
        nb = n_bins or n // 2
        k, pk, dpk = np.zeros((self.B, nb)), np.zeros((self.B, nb)), np.zeros((self.B, nb))
        cnt = np.zeros((self.B, nb), dtype=np.int64)
        self._stream()
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._check(self.lib.pm_power_spectrum_jvp(self.h, _ptr(disp), _ptr(tdisp), int(n), int(nb), dptr(k), dptr(pk),
                                                   dptr(dpk), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return k, pk, dpk, cnt

    def ic_adjoint(self, noise, adj_disp, adj_vel, with_sigma8=True):
        out = torch.empty((self.B, self.N), device=self.device, dtype=torch.float32)
        ds8 = np.zeros(self.B)
        self._stream()
        self._check(self.lib.pm_ic_adjoint(self.h, _ptr(noise), _ptr(adj_disp), _ptr(adj_vel), _ptr(out),
                                           ds8.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if with_sigma8
                                           else None))
        return out, (ds8 if with_sigma8 else None)

    def density_vjp(self, disp, ddelta, n_mesh=None, order=None):
        n = n_mesh or self.cfg.n_mesh
        self._state_ok(ddelta, "dL_ddelta", (self.B, n, n, n))
        out = torch.empty((self.B, 3, self.N), device=self.device, dtype=torch.float32)
        self._stream()
        self._check(self.lib.pm_density_vjp(self.h, _ptr(disp), int(n), int(order or self.cfg.order), _ptr(ddelta),
                                            _ptr(out)))
        return out

    PHASES = ("deposit", "fft_x_fwd", "fft_y_fwd", "fft_z_green", "fft_y_inv", "fft_x_inv",
              "interp_kick_drift", "ic_zeldovich", "power_spectrum", "adjoint_spectral", "reserved",
              "grad_stencil")

    def profile(self, enable=True):
        self._check(self.lib.pm_profile(self.h, int(bool(enable))))

    def profile_read(self):
        ms = np.zeros(12)
        calls = np.zeros(12, dtype=np.int64)
        launches = np.zeros(12, dtype=np.int64)
        self._check(self.lib.pm_profile_read(self.h, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             calls.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                             launches.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 12))
        return {p: dict(ms=ms[i], calls=int(calls[i]), launches=int(launches[i])) for i, p in enumerate(self.PHASES)}

    def simulate_host(self, noise, disp=None, vel=None):
        """noise: host float32 array/tensor [B, N] (pinned for full speed); returns host disp, vel."""
        if isinstance(noise, np.ndarray):
            noise = torch.from_numpy(np.ascontiguousarray(noise, dtype=np.float32))
        if disp is None:
            disp = torch.empty((self.B, 3, self.N), dtype=torch.float32, pin_memory=True)
            vel = torch.empty((self.B, 3, self.N), dtype=torch.float32, pin_memory=True)
        self._stream()
        self._check(self.lib.pm_simulate_host(self.h, ctypes.c_void_p(noise.data_ptr()),
                                              ctypes.c_void_p(disp.data_ptr()), ctypes.c_void_p(vel.data_ptr())))
        return disp, vel

    def simulate_pk_host(self, noise, n_mesh=None, n_bins=None):
        """noise: host float32 array/tensor [B, N] (pinned for full speed).  ICs, the
        whole run and the power spectrum of the final positions; returns host
        (k, P, counts) [B, n_bins].  The state stays in the handle's device buffers."""
        if isinstance(noise, np.ndarray):
            noise = torch.from_numpy(np.ascontiguousarray(noise, dtype=np.float32))
        if noise.is_cuda or noise.dtype != torch.float32 or not noise.is_contiguous() or \
                noise.numel() != self.B * self.N:
            raise ValueError(f"noise must be a contiguous float32 host tensor of {self.B} x {self.N} values")
        n = n_mesh or (self.cfg.pk_mesh_max or self.cfg.n_mesh)
        nb = n_bins or n // 2
        k, pk = np.zeros((self.B, nb)), np.zeros((self.B, nb))
        cnt = np.zeros((self.B, nb), dtype=np.int64)
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._stream()
        self._check(self.lib.pm_simulate_pk_host(self.h, ctypes.c_void_p(noise.data_ptr()), int(n), int(nb), dptr(k),
                                                 dptr(pk), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return k, pk, cnt


def power_spectrum_static(disp, n_part, box, n_mesh, n_bins, stream=None):
    """pm_power_spectrum_static: P(k) of one simulation without any device
    allocation (fixed scratch inside the library, n_mesh <= 64)."""
    lib = _lib.load()
    k = np.zeros(n_bins)
    pk = np.zeros(n_bins)
    cnt = np.zeros(n_bins, dtype=np.int64)
    s = stream if stream is not None else torch.cuda.current_stream(disp.device).cuda_stream
    rc = lib.pm_power_spectrum_static(ctypes.c_void_p(disp.data_ptr()), int(n_part), float(box), int(n_mesh),
                                      int(n_bins), ctypes.c_void_p(s),
                                      k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      pk.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    _lib.check(rc)
    return k, pk, cnt
