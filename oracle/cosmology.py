"""Oracle cosmology: growth functions, kick coefficients, linear spectrum.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions
-----------
* Flat LambdaCDM without radiation: (H/H0)^2 = Omega_m a^-3 + Omega_L,
  Omega_L = 1 - Omega_m (the paper restricts itself to flat cosmologies, Sec. 3.1).
* D is normalised as D ~ a for a -> 0 and E ~ -(3/7) D^2, which is the
  normalisation the BullFrog coefficients use (Sec. 2.4, footnote on the growth
  factor).
"""
import math

import numpy as np
from scipy import integrate


def hubble2(a, omega_m):
    """(H(a)/H0)^2 for flat LambdaCDM (Eq. poisson context, Sec. 2)."""
    return omega_m / a ** 3 + (1.0 - omega_m)


def gamma(a, omega_m):
    """gamma = Omega_m H0^2 / (2 a^3 H^2)  (App. B, definition under Eq. growth_odes)."""
    return omega_m / (2.0 * a ** 3 * hubble2(a, omega_m))


def dlnH_dlna(a, omega_m):
    """d ln H / d ln a, differentiated by hand from ``hubble2``."""
    return 0.5 * (-3.0 * omega_m / a ** 3) / hubble2(a, omega_m)


class Growth:
    """First- and second-order growth D(a), E(a) (App. B, Eq. growth_odes).

    Reading: the printed friction term of the growth-rate equations,
    -d(1 - gamma), only agrees with the standard linear growth equation
    D'' + (2 + dlnH/dlna) D' = 3 gamma D in Einstein-de Sitter.  We take the
    standard form (friction 2 + dlnH/dlna = 2 - 3 gamma for flat LambdaCDM),
    which is pinned against the closed-form integral solution for D in
    ``tests/test_oracle_cosmology.py``.  Written as second-order ODEs in ln a
    for (D, dD/dlna) and (E, dE/dlna):

        D''  = 3 gamma D            - (2 + dlnH/dlna) D'
        E''  = 3 gamma (E - D^2)    - (2 + dlnH/dlna) E'

    (dividing by D resp. E and substituting d = D'/D, e = E'/E gives the
    App. B equations for the growth rates).  Integrated with classical RK4 at
    uniform steps in ln a (App. B: "a simple Runge-Kutta integrator with
    uniform steps in ln a"), started at a0 on the EdS growing mode
    D = a, E = -(3/7) a^2.
    """

    def __init__(self, omega_m, a0=1e-4, a_max=2.0, h=1e-3):
        self.omega_m = float(omega_m)
        self.h = h
        self.lna0 = math.log(a0)
        nstep = int(math.ceil((math.log(a_max) - self.lna0) / h))
        self.lna = self.lna0 + h * np.arange(nstep + 1)
        y = np.array([a0, a0, -3.0 / 7.0 * a0 ** 2, -6.0 / 7.0 * a0 ** 2])
        ys = np.empty((nstep + 1, 4))
        ys[0] = y
        for i in range(nstep):
            y = self._rk4(self.lna[i], y, h)
            ys[i + 1] = y
        self.ys = ys

    def _rhs(self, lna, y):
        a = math.exp(lna)
        g = gamma(a, self.omega_m)
        fr = 2.0 + dlnH_dlna(a, self.omega_m)
        D, dD, E, dE = y
        return np.array([dD, 3.0 * g * D - fr * dD, dE, 3.0 * g * (E - D * D) - fr * dE])

    def _rk4(self, x, y, h):
        k1 = self._rhs(x, y)
        k2 = self._rhs(x + 0.5 * h, y + 0.5 * h * k1)
        k3 = self._rhs(x + 0.5 * h, y + 0.5 * h * k2)
        k4 = self._rhs(x + h, y + h * k3)
        return y + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)

    def state(self, a):
        """(D, dD/dlna, E, dE/dlna) at a: one RK4 step from the grid node below."""
        lna = math.log(a)
        i = int((lna - self.lna0) // self.h)
        i = min(max(i, 0), len(self.lna) - 2)
        dx = lna - self.lna[i]
        if dx == 0.0:
            return self.ys[i].copy()
        return self._rk4(self.lna[i], self.ys[i], dx)

    def D(self, a):
        return self.state(a)[0]

    def E(self, a):
        return self.state(a)[2]

    def dE_dD(self, a):
        """E'(D) = dE/dD = (dE/dlna) / (dD/dlna)  (derivative w.r.t. D, Sec. 2.4)."""
        s = self.state(a)
        return s[3] / s[1]

    def dD_dlna(self, a):
        return self.state(a)[1]

    def a_of_D(self, D):
        """Inverse of D(a) by bisection (D is monotonic in a)."""
        lo, hi = math.exp(self.lna0), math.exp(self.lna[-1])
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if self.D(mid) < D:
                lo = mid
            else:
                hi = mid
            if hi - lo < 1e-15 * hi:
                break
        return 0.5 * (lo + hi)


def step_table(growth, a_ini, a_end, n_steps, stepper="bullfrog", time_var="D"):
    """Per-step DKD coefficients (tau1, tau2, alpha, beta, D_half, D_n, D_{n+1}).

    Sec. 2.4 / Eq. dkd: X_half = X + tau1 V; V' = alpha V + beta A(X_half);
    X' = X_half + tau2 V'.  Velocities are D-time velocities V = dX/dD.

    time_var "D": D_n = D_0 + n dD and D_half = D_0 + (n + 1/2) dD.
    time_var "a": a_n = a_0 + n da, a_half = a_0 + (n + 1/2) da and D_half = D(a_half).
    In both cases tau1 = D_half - D_n and tau2 = D_{n+1} - D_half.

    BullFrog (Sec. 2.4): alpha = (E'(D_{n+1}) - xi) / (E'(D_n) - xi),
    beta = (1 - alpha) D_half, with
    xi = (E_n + E'(D_n) tau1) / D_half - D_half.
    Reading: the paper prints E'(D_n) (D_{n+1} - D_n)/2 in xi, which equals
    E'(D_n) tau1 for steps centred in D; we write tau1 so that steps centred in
    another variable stay 2LPT-consistent (pinned by the mock-2LPT stepper
    test).

    FastPM (Sec. 2.4): alpha = zeta(a_n) / zeta(a_{n+1}), zeta = H a^3 dD/da,
    beta = (1 - alpha) D_half.
    """
    rows = []
    if time_var == "D":
        D0, D1 = growth.D(a_ini), growth.D(a_end)
        dD = (D1 - D0) / n_steps
        Dn = [D0 + i * dD for i in range(n_steps + 1)]
        Dh = [D0 + (i + 0.5) * dD for i in range(n_steps)]
        an = [growth.a_of_D(d) for d in Dn]
        an[0], an[-1] = a_ini, a_end
    elif time_var == "a":
        da = (a_end - a_ini) / n_steps
        an = [a_ini + i * da for i in range(n_steps + 1)]
        an[-1] = a_end
        Dn = [growth.D(a) for a in an]
        Dh = [growth.D(a_ini + (i + 0.5) * da) for i in range(n_steps)]
    else:
        raise ValueError(time_var)
    for i in range(n_steps):
        tau1 = Dh[i] - Dn[i]
        tau2 = Dn[i + 1] - Dh[i]
        if stepper == "bullfrog":
            En = growth.E(an[i])
            Epn = growth.dE_dD(an[i])
            Epn1 = growth.dE_dD(an[i + 1])
            xi = (En + Epn * tau1) / Dh[i] - Dh[i]
            alpha = (Epn1 - xi) / (Epn - xi)
        elif stepper == "fastpm":
            def zeta(a):
                # H a^3 dD/da = H a^2 dD/dlna (H in units of H0; the ratio is unit-free)
                return math.sqrt(hubble2(a, growth.omega_m)) * a ** 2 * growth.dD_dlna(a)
            alpha = zeta(an[i]) / zeta(an[i + 1])
        else:
            raise ValueError(stepper)
        beta = (1.0 - alpha) * Dh[i]
        rows.append((tau1, tau2, alpha, beta, Dh[i], Dn[i], Dn[i + 1]))
    return np.array(rows)


# --- linear power spectrum (not in the paper: BBKS stands in for the
#     Einstein-Boltzmann module; Bardeen, Bond, Kaiser & Szalay 1986, App. G) ---

def bbks_transfer(k, omega_m, h):
    """BBKS transfer function, shape parameter Gamma = Omega_m h (no baryon
    correction; k in h/Mpc, q = k / Gamma)."""
    k = np.asarray(k, dtype=np.float64)
    q = k / (omega_m * h)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.log1p(2.34 * q) / (2.34 * q) * (
            1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25
    return np.where(q > 0, t, 1.0)


def tophat_window(x):
    """Fourier transform of a spherical top-hat, 3 (sin x - x cos x) / x^3."""
    x = np.asarray(x, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        w = 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3
    return np.where(x > 1e-4, w, 1.0 - x * x / 10.0)


def sigma_r(pk_fn, R=8.0):
    """sigma_R^2 = 1/(2 pi^2) int k^2 P(k) W(kR)^2 dk, integrated in ln k by quad."""
    def integrand(lnk):
        k = math.exp(lnk)
        return k ** 3 * pk_fn(k) * float(tophat_window(k * R)) ** 2 / (2.0 * math.pi ** 2)
    val, _ = integrate.quad(integrand, math.log(1e-6), math.log(1e3), limit=2000,
                            epsabs=0.0, epsrel=1e-12)
    return math.sqrt(val)


class LinearSpectrum:
    """P_lin(k, a=1) = A k^n_s T_BBKS(k)^2, with A fixed so that sigma_8 = sigma8."""

    def __init__(self, omega_m, h, n_s, sigma8):
        self.omega_m, self.hh, self.n_s, self.sigma8 = omega_m, h, n_s, sigma8
        self.A = 1.0
        s = sigma_r(self.__call__, 8.0)
        self.A = (sigma8 / s) ** 2

    def __call__(self, k):
        k = np.asarray(k, dtype=np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            p = self.A * np.power(k, self.n_s) * bbks_transfer(k, self.omega_m, self.hh) ** 2
        return np.where(k > 0, p, 0.0)
