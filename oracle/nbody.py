"""Oracle N-body: Zel'dovich ICs, the DKD/BullFrog PM stepper and its adjoint.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

State: displacements Psi = X - q and D-time velocities V = dX/dD, both arrays
of shape (3, N), particle i = (iz n + iy) n + ix on the Lagrangian lattice
q = (ix, iy, iz) L / n_p (reading: the paper does not place the lattice; the
corner placement makes an unperturbed lattice deposit a uniform density).
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import cosmology, mesh


@dataclass
class Config:
    n_part: int
    n_mesh: int
    box: float
    order: int = 2              # 2 = CIC, 3 = TSC, 4 = PCS (Table 1)
    interlace: bool = False
    grad_order: int = 4         # Table 4 default
    lap_order: int = 0          # Table 4 default
    omega_m: float = 0.3
    h: float = 0.7
    n_s: float = 0.96
    sigma8: float = 0.8
    a_ini: float = 0.02
    a_end: float = 1.0
    n_steps: int = 6
    stepper: str = "bullfrog"
    time_var: str = "D"
    zero_corner: bool = True
    deconvolve: bool = False    # divide the force's density by the squared kernel (Table 4 `deconvolve`)
    lpt_order: int = 1          # 1 = Zel'dovich ICs, 2 = 2LPT ICs (Table 4 `nlpt_order_ics`)
    nufft: bool = False         # force by the NUFFT on the n_mesh band (Sec. 2.5; ES kernel, grid 2 n_mesh)
    growth: object = field(default=None, repr=False)

    @property
    def deconv_order(self):
        return self.order if self.deconvolve else 0

    def get_growth(self):
        if self.growth is None:
            self.growth = cosmology.Growth(self.omega_m)
        return self.growth


def lattice(n, L):
    """Lagrangian positions q, shape (3, n^3), x fastest."""
    i = np.arange(n) * (L / n)
    qz, qy, qx = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([qx.reshape(-1), qy.reshape(-1), qz.reshape(-1)])


# --------------------------------------------------------------------------
# initial conditions (Sec. 2.2, Zel'dovich approximation; Sec. 2.4)
# --------------------------------------------------------------------------

def ic_multipliers(cfg, pk=None):
    """Fourier multipliers mIC_c with psi1_c^ = mIC_c w^ for white noise w.

    delta_lin(a=1)^ = w^ sqrt(P(k) n^3 / L^3)  (unit-variance white noise);
    psi1^ = i k / k^2 delta_lin^ / D(1) in the D ~ a normalisation, so that
    X = q + D psi1 has linear density -D div psi1 = delta_lin D / D(1).
    Zeroed: k = 0, every Nyquist plane, and (if zero_corner, Table 4 caption:
    corner modes are zeroed by default; App. A.3) every |k| > k_Ny.
    """
    n, L = cfg.n_part, cfg.box
    pk = pk or cosmology.LinearSpectrum(cfg.omega_m, cfg.h, cfg.n_s, cfg.sigma8)
    D1 = cfg.get_growth().D(1.0)
    k1 = mesh.wavenumbers(n, L)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    kmag = np.sqrt(k2)
    amp = np.sqrt(pk(kmag) * n ** 3 / L ** 3)
    nyq = np.arange(n) == n // 2
    nz, ny, nx = np.meshgrid(nyq, nyq, nyq, indexing="ij")
    keep = ~(nx | ny | nz) & (k2 > 0)
    if cfg.zero_corner:
        keep &= kmag <= math.pi * n / L
    with np.errstate(divide="ignore", invalid="ignore"):
        base = np.where(keep, amp / np.where(k2 > 0, k2, 1.0) / D1, 0.0)
    return [1j * kc * base for kc in (kx, ky, kz)]


def lpt2_term(psi1, L):
    """Second-order LPT displacement psi^(2) of Eq. LPT from the first-order one
    (Sec. 2.2, Eqs. helmholtz / LPT_L_and_T / LPT_kernels at n = 2, D^n growth).

    At n = 2 the transverse part vanishes (the factor n - 2s is zero for s = 1) and
    the longitudinal part is L^(2) = -(3/7) mu_2L^(1,1) with
    mu_2L^(1,1) = (1/2)(psi_i,i psi_j,j - psi_i,j psi_j,i) (sums over i, j); then
    psi^(2) = Lap^-1 grad L^(2).  Derivatives and the inverse Laplacian use the
    exact kernels i k and -k^2 (as the paper states for LPT).  Readings: the
    products are formed on the n^3 grid without the 3/2-rule padding, and psi^(2)
    is zeroed at k = 0 and on every Nyquist plane, like psi^(1).
    psi1: (3, n^3) real; returns (3, n^3)."""
    n = round(psi1.shape[1] ** (1.0 / 3.0))
    k1 = mesh.wavenumbers(n, L)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = (kx, ky, kz)
    ph = [np.fft.fftn(psi1[c].reshape(n, n, n)) for c in range(3)]
    # d[i][j] = d psi_i / d q_j
    d = [[np.fft.ifftn(1j * kk[j] * ph[i]).real for j in range(3)] for i in range(3)]
    mu2 = np.zeros((n, n, n))
    for i in range(3):
        for j in range(3):
            mu2 += 0.5 * (d[i][i] * d[j][j] - d[i][j] * d[j][i])
    L2 = -3.0 / 7.0 * mu2
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    nyq = np.arange(n) == n // 2
    nz, ny, nx = np.meshgrid(nyq, nyq, nyq, indexing="ij")
    keep = ~(nx | ny | nz) & (k2 > 0)
    L2k = np.fft.fftn(L2)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(keep, -1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    return np.stack([np.fft.ifftn(1j * kc * inv * L2k).real.reshape(-1) for kc in kk])


def zeldovich_ic(cfg, w, pk=None):
    """Psi0 = D(a_ini) psi1, V0 = psi1 from white noise w (shape (n,n,n), [z,y,x]).
    With cfg.lpt_order = 2 (2LPT, Eq. LPT truncated at n = 2 with D^n growth):
    Psi0 = D psi1 + D^2 psi2 and V0 = dPsi/dD = psi1 + 2 D psi2."""
    ms = ic_multipliers(cfg, pk)
    psi1 = np.stack([mesh.apply_multiplier(w, m).reshape(-1) for m in ms])
    Dini = cfg.get_growth().D(cfg.a_ini)
    if cfg.lpt_order == 2:
        psi2 = lpt2_term(psi1, cfg.box)
        return Dini * psi1 + Dini ** 2 * psi2, psi1 + 2.0 * Dini * psi2
    return Dini * psi1, psi1.copy()


# --------------------------------------------------------------------------
# force at the particles (Sec. 2.5)
# --------------------------------------------------------------------------

def nufft_band_force(X, n, L):
    """Force at the particles from the non-uniform DFT of their positions,
    restricted to the band of an n^3 mesh (Sec. 2.5, force evaluation with the
    non-uniform FFT): delta^(k) = (M/N) sum_i exp(-i k.X_i) for the modes with
    |m_c| < n/2 on every axis (k != 0; M = n^3), g_c^ = m_c delta^ with the exact
    multiplier m_c = -i k_c / (-k^2), and g_c(X_i) = (1/M) sum_k g_c^(k) exp(i k.X_i)
    evaluated exactly at each particle.  This is the plain definition that a
    NUFFT approximates to its kernel's accuracy.  X: (3, N); returns (3, N)."""
    N = X.shape[1]
    M = n ** 3
    m1 = np.arange(-(n // 2) + 1, n // 2)
    mz, my, mx = np.meshgrid(m1, m1, m1, indexing="ij")
    kv = 2.0 * math.pi / L * np.stack([mx.reshape(-1), my.reshape(-1), mz.reshape(-1)])   # (3, K)
    k2 = (kv ** 2).sum(axis=0)
    keep = k2 > 0
    kv, k2 = kv[:, keep], k2[keep]
    dk = np.zeros(kv.shape[1], dtype=complex)
    for c0 in range(0, N, 2048):
        ph = kv.T @ X[:, c0:c0 + 2048]                  # (K, chunk)
        dk += np.exp(-1j * ph).sum(axis=1)
    dk *= M / N
    out = np.zeros((3, N))
    for c in range(3):
        gk = (1j * kv[c] / k2) * dk                     # -(i k_c) / (-k^2) delta^
        for c0 in range(0, N, 2048):
            ph = kv.T @ X[:, c0:c0 + 2048]
            out[c, c0:c0 + 2048] = (gk[:, None] * np.exp(1j * ph)).sum(axis=0).real / M
    return out


def accel(cfg, Psi, q, Dh):
    """A(X) = g(X) / D_half^2 with g = -grad Lap^-1 delta (units of length).

    Reading (the paper never normalises A): with D-time velocities and
    beta = (1 - alpha) D_half, Zel'dovich consistency (V stays psi1 under the
    linear force g = D psi1) needs A = g / D_half^2; pinned by the plane-wave
    and mock-force tests.

    Interlacing (Sec. 2.8, one extra grid): the second grid deposits X + s,
    s = (H/2)(1,1,1); delta^ = (delta0^ + e^{ik.s} delta1^)/2; the force
    spectrum g^ is brought back on both grids (g^ and g^ e^{-ik.s}), each is
    interpolated at its own offset, and the two are averaged.  Every mode on a
    Nyquist plane is zeroed in that case.
    """
    n, L = cfg.n_mesh, cfg.box
    X = np.mod(q + Psi, L)
    if cfg.nufft:
        return mesh.nufft_force(X, n, L) / Dh ** 2
    if not cfg.interlace:
        delta = mesh.density_contrast(X, n, L, cfg.order)
        g = mesh.force_field(delta, L, cfg.grad_order, cfg.lap_order, cfg.deconv_order)
        A = np.stack([mesh.gather(gc, X, L, cfg.order) for gc in g])
    else:
        H = L / n
        s = 0.5 * H
        d0 = np.fft.fftn(mesh.density_contrast(X, n, L, cfg.order))
        d1 = np.fft.fftn(mesh.density_contrast(X, n, L, cfg.order, shift=s))
        dk = 0.5 * (d0 + mesh.interlace_phase(n, L, +1) * d1)
        ms = mesh.force_multipliers(n, L, cfg.grad_order, cfg.lap_order, zero_all_nyquist=True,
                                    deconvolve_order=cfg.deconv_order)
        back = mesh.interlace_phase(n, L, -1)
        A = []
        for m in ms:
            g0 = np.fft.ifftn(m * dk).real
            g1 = np.fft.ifftn(m * dk * back).real
            A.append(0.5 * (mesh.gather(g0, X, L, cfg.order) + mesh.gather(g1, X, L, cfg.order, shift=s)))
        A = np.stack(A)
    return A / Dh ** 2


# --------------------------------------------------------------------------
# DKD stepper (Eq. dkd)
# --------------------------------------------------------------------------

def step(cfg, Psi, V, coef, q, force_fn=None):
    """One DKD step: X_half = X + tau1 V; V' = alpha V + beta A(X_half);
    X' = X_half + tau2 V'.  ``force_fn(Psi_half, D_half)`` replaces the PM
    force (used by the mock-force pins)."""
    tau1, tau2, alpha, beta, Dh = coef[:5]
    Ph = Psi + tau1 * V
    A = force_fn(Ph, Dh) if force_fn else accel(cfg, Ph, q, Dh)
    V2 = alpha * V + beta * A
    return Ph + tau2 * V2, V2


def run(cfg, Psi, V, table=None, force_fn=None, n_steps=None):
    table = cosmology.step_table(cfg.get_growth(), cfg.a_ini, cfg.a_end, cfg.n_steps,
                                 cfg.stepper, cfg.time_var) if table is None else table
    q = lattice(cfg.n_part, cfg.box)
    for row in table[: (n_steps or len(table))]:
        Psi, V = step(cfg, Psi, V, row, q, force_fn)
    return Psi, V


# --------------------------------------------------------------------------
# forward mode (tangents; the JVP counterpart of App. C)
# --------------------------------------------------------------------------

def accel_jvp(cfg, Psi_h, q, Dh, T):
    """(grad_X A) . T for A = g(X)/Dh^2 (non-interlaced PM): returns (3, N).

    A_kc = Dh^-2 sum_j g_cj W(r_j - X_k), g_c = F_c delta, delta = (M/N) scatter(1) - 1.
    Two contributions: the gather's dependence on the positions,
    sum_d T_dk sum_j g_cj dW/dX_dk; and on the mesh, the gather of
    g'_c = F_c delta', delta' = (M/N) scatter_dot_grad(T)."""
    if cfg.interlace:
        raise NotImplementedError("forward mode is defined for a single grid")
    n, L = cfg.n_mesh, cfg.box
    N = Psi_h.shape[1]
    X = np.mod(q + Psi_h, L)
    delta = mesh.density_contrast(X, n, L, cfg.order)
    ms = mesh.force_multipliers(n, L, cfg.grad_order, cfg.lap_order, deconvolve_order=cfg.deconv_order)
    g = [mesh.apply_multiplier(delta, m) for m in ms]
    ddelta = (n ** 3 / N) * mesh.scatter_dot_grad(X, T, n, L, cfg.order)
    out = np.zeros((3, N))
    for c in range(3):
        gg = mesh.gather_grad(g[c], X, L, cfg.order)
        out[c] = (T * gg).sum(axis=0) + mesh.gather(mesh.apply_multiplier(ddelta, ms[c]), X, L, cfg.order)
    return out / Dh ** 2


def step_jvp(cfg, Psi, V, Pt, Vt, coef, q):
    """One DKD step with its tangent: (Psi, V, Psi', V') -> the next state and tangent."""
    tau1, tau2, alpha, beta, Dh = coef[:5]
    Ph, Pht = Psi + tau1 * V, Pt + tau1 * Vt
    A = accel(cfg, Ph, q, Dh)
    At = accel_jvp(cfg, Ph, q, Dh, Pht)
    V2, V2t = alpha * V + beta * A, alpha * Vt + beta * At
    return Ph + tau2 * V2, V2, Pht + tau2 * V2t, V2t


def run_jvp(cfg, Psi, V, Pt, Vt, table=None):
    table = cosmology.step_table(cfg.get_growth(), cfg.a_ini, cfg.a_end, cfg.n_steps,
                                 cfg.stepper, cfg.time_var) if table is None else table
    q = lattice(cfg.n_part, cfg.box)
    for row in table:
        Psi, V, Pt, Vt = step_jvp(cfg, Psi, V, Pt, Vt, row, q)
    return Psi, V, Pt, Vt


def power_spectrum_jvp(Psi, Pt, n, L, n_bins, order=2):
    """Tangent of the binned P(k) of the CIC density of X = q + Psi along Psi':
    P_b = (L^3/M^2) <|delta^|^2>_b, so P'_b = (L^3/M^2) <2 Re(conj(delta^) delta'^)>_b with
    delta' = (M/N) scatter_dot_grad(Psi').  Returns (k_mean, P', counts)."""
    N = Psi.shape[1]
    npart = round(N ** (1.0 / 3.0))
    X = np.mod(lattice(npart, L) + Psi, L)
    delta = mesh.density_contrast(X, n, L, order)
    dt = (n ** 3 / N) * mesh.scatter_dot_grad(X, Pt, n, L, order)
    dk, dtk = np.fft.fftn(delta), np.fft.fftn(dt)
    k1 = mesh.wavenumbers(n, L)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    kF = 2 * math.pi / L
    b = np.floor(kmag / kF - 0.5).astype(np.int64)
    ok = (kmag > 0) & (b >= 0) & (b < n_bins)
    cross = 2.0 * (np.conj(dk) * dtk).real
    cnt = np.bincount(b[ok], minlength=n_bins)[:n_bins]
    ksum = np.bincount(b[ok], weights=kmag[ok], minlength=n_bins)[:n_bins]
    psum = np.bincount(b[ok], weights=cross[ok], minlength=n_bins)[:n_bins]
    M = n ** 3
    with np.errstate(invalid="ignore", divide="ignore"):
        return (np.where(cnt > 0, ksum / np.maximum(cnt, 1), 0.0),
                np.where(cnt > 0, psum / np.maximum(cnt, 1) * L ** 3 / M ** 2, 0.0), cnt)


# --------------------------------------------------------------------------
# adjoint (Sec. 2.7, Table 5; App. C)
# --------------------------------------------------------------------------

def accel_vjp(cfg, Psi_h, q, Dh, u):
    """u . grad_X A(X)  for A = g(X)/Dh^2 (non-interlaced PM): returns (3, N).

    A_kc = Dh^-2 sum_j g_cj W(r_j - X_k), g_c = F_c delta, delta = (M/N) scatter(1) - 1.
    Two contributions (App. C table):
      * gather w.r.t. positions: -> sum_c u_kc sum_j g_cj dW/dX_k (gather with grad W);
      * gather w.r.t. mesh: s_c = scatter(u_c) (scatter with W), then the mesh
        cotangent of delta is rho~ = sum_c F_c^T s_c, where F_c^T has the
        multiplier conj(m_c); then scatter w.r.t. positions:
        -> (M/N) sum_j rho~_j dW/dX_i (gather of rho~ with grad W).
    """
    if cfg.interlace:
        raise NotImplementedError("adjoint is defined for a single grid")
    n, L = cfg.n_mesh, cfg.box
    N = Psi_h.shape[1]
    X = np.mod(q + Psi_h, L)
    delta = mesh.density_contrast(X, n, L, cfg.order)
    ms = mesh.force_multipliers(n, L, cfg.grad_order, cfg.lap_order, deconvolve_order=cfg.deconv_order)
    g = [mesh.apply_multiplier(delta, m) for m in ms]
    out = np.zeros((3, N))
    for c in range(3):
        out += u[c] * mesh.gather_grad(g[c], X, L, cfg.order)
    rho_t = np.zeros((n, n, n))
    for c in range(3):
        s_c = mesh.scatter(X, u[c], n, L, cfg.order)
        rho_t += mesh.apply_multiplier(s_c, np.conj(ms[c]))
    out += (n ** 3 / N) * mesh.gather_grad(rho_t, X, L, cfg.order)
    return out / Dh ** 2


def adjoint(cfg, Psi, V, Xa, Va, table=None):
    """Backward-in-time DKD for (X, V, X*, V*) (Table 5), memory O(1) in steps.

    Per step n (reversed):
      X_half = X - tau2 V;  V* += tau2 X*;
      V_prev = (V - beta A(X_half)) / alpha;  X* += beta V*.grad A(X_half);
      V* = alpha V*;  X = X_half - tau1 V_prev;  V* += tau1 X*.
    Returns the reintegrated initial state and the cotangents (Psi0, V0, X*0, V*0).
    """
    table = cosmology.step_table(cfg.get_growth(), cfg.a_ini, cfg.a_end, cfg.n_steps,
                                 cfg.stepper, cfg.time_var) if table is None else table
    q = lattice(cfg.n_part, cfg.box)
    Xa, Va = Xa.copy(), Va.copy()
    for row in table[::-1]:
        tau1, tau2, alpha, beta, Dh = row[:5]
        Ph = Psi - tau2 * V
        Va = Va + tau2 * Xa
        A = accel(cfg, Ph, q, Dh)
        Vp = (V - beta * A) / alpha
        Xa = Xa + beta * accel_vjp(cfg, Ph, q, Dh, Va)
        Va = alpha * Va
        Psi = Ph - tau1 * Vp
        V = Vp
        Va = Va + tau1 * Xa
    return Psi, V, Xa, Va


def ic_vjp(cfg, Xa0, Va0, w, pk=None):
    """Pull (X*0, V*0) back through Psi0 = D_ini psi1, V0 = psi1, psi1 = F_IC w.

    psi1* = D_ini X*0 + V*0; w* = sum_c F_IC,c^T psi1*_c (multiplier conj(mIC_c));
    sigma8 enters only as an overall factor of psi1, so dL/dsigma8 = <psi1*, psi1> / sigma8.
    """
    n = cfg.n_part
    Dini = cfg.get_growth().D(cfg.a_ini)
    ps = Dini * Xa0 + Va0
    ms = ic_multipliers(cfg, pk)
    wa = np.zeros((n, n, n))
    for c in range(3):
        wa += mesh.apply_multiplier(ps[c].reshape(n, n, n), np.conj(ms[c]))
    psi1 = np.stack([mesh.apply_multiplier(w, m).reshape(-1) for m in ms])
    ds8 = float(np.sum(ps * psi1)) / cfg.sigma8
    return wa, ds8


def density_vjp(cfg, Psi, dL_ddelta, n=None, order=None):
    """Cotangent of final positions from dL/d delta of delta = (M/N) scatter(1) - 1
    (App. C: VJP of scatter w.r.t. positions is a gather with grad W)."""
    n = n or cfg.n_mesh
    order = order or cfg.order
    N = Psi.shape[1]
    X = np.mod(lattice(cfg.n_part, cfg.box) + Psi, cfg.box)
    return (n ** 3 / N) * mesh.gather_grad(dL_ddelta, X, cfg.box, order)
