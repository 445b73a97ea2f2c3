"""Pins of the oracle's cosmology (growth ODE, kick coefficients, BBKS, sigma8)
against closed forms and numbers printed in the paper (App. B, Sec. 2.4)."""
import math
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest
from scipy import integrate

from oracle import cosmology, nbody

GOLDEN = Path(__file__).parent / "golden"


def _paper_constants():
    out = {}
    for line in (GOLDEN / "paper_constants.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(Fraction(v))
    return out


def test_eds_growth_closed_form():
    # Omega_m = 1: D = a and E = -(3/7) a^2 exactly (EdS growing modes).
    g = cosmology.Growth(1.0)
    for a in (0.01, 0.02, 0.3, 1.0):
        assert g.D(a) == pytest.approx(a, rel=1e-11)
        assert g.E(a) == pytest.approx(-3.0 / 7.0 * a * a, rel=1e-10)
        assert g.dE_dD(a) == pytest.approx(-6.0 / 7.0 * a, rel=1e-10)


@pytest.mark.parametrize("om", [0.3, 0.3158])
def test_lcdm_growth_matches_integral_solution(om):
    # Closed form of the growing mode for dust + Lambda (Heath 1977):
    # D(a) = (5 Om / 2) H(a)/H0 int_0^a da' / (a' H(a')/H0)^3,  normalised to D ~ a.
    g = cosmology.Growth(om)
    for a in (0.02, 0.1, 0.5, 1.0):
        E = math.sqrt(cosmology.hubble2(a, om))
        val, _ = integrate.quad(lambda x: 1.0 / (x * math.sqrt(cosmology.hubble2(x, om))) ** 3,
                                0.0, a, epsabs=0, epsrel=1e-13, limit=500)
        D_exact = 2.5 * om * E * val
        assert g.D(a) == pytest.approx(D_exact, rel=1e-9)


def test_second_order_growth_series():
    # Sec. 2.4: E = -(3/7) D^2 - (3/1001) Lambda D^5 + O(Lambda^2 D^8).
    c = _paper_constants()
    om = 0.3
    lam = (1 - om) / om
    g = cosmology.Growth(om)
    for a in (0.01, 0.02, 0.05):
        D = g.D(a)
        series = c["E_series_D2"] * D ** 2 + c["E_series_D5"] * lam * D ** 5
        # the O(Lambda^2 D^8) remainder is ~ Lambda^2 D^8; the D^5 term itself is
        # ~1e-7 relative, so a tolerance of 1e-9 checks it.
        assert g.E(a) == pytest.approx(series, rel=max(1e-11, 5 * lam ** 2 * D ** 6))
    # the D^5 term matters: dropping it fails at a = 0.05
    D = g.D(0.05)
    assert abs(g.E(0.05) - c["E_series_D2"] * D ** 2) > 1e-3 * abs(c["E_series_D5"] * lam * D ** 5) * 100


def test_fastpm_alpha_eds_closed_form():
    # EdS: zeta = H a^3 dD/da = a^{3/2}, so alpha = (a_n / a_{n+1})^{3/2}.
    g = cosmology.Growth(1.0)
    tab = cosmology.step_table(g, 0.1, 1.0, 4, stepper="fastpm", time_var="a")
    an = np.linspace(0.1, 1.0, 5)
    for i, row in enumerate(tab):
        assert row[2] == pytest.approx((an[i] / an[i + 1]) ** 1.5, rel=1e-9)
        assert row[3] == pytest.approx((1 - row[2]) * row[4], rel=1e-12)


@pytest.mark.parametrize("time_var", ["D", "a"])
@pytest.mark.parametrize("om", [1.0, 0.3])
def test_zeldovich_consistency_mock_linear_force(om, time_var):
    # Sec. 2.4: with beta = (1 - alpha) D_half, a linear force g = a psi1 keeps
    # V = psi1 and X = q + D psi1 exactly after every step (any alpha).
    cfg = nbody.Config(n_part=1, n_mesh=1, box=1.0, omega_m=om, a_ini=0.02, a_end=1.0,
                       n_steps=5, time_var=time_var)
    g = cfg.get_growth()
    tab = cosmology.step_table(g, cfg.a_ini, cfg.a_end, cfg.n_steps, "bullfrog", time_var)
    psi1 = np.array([[0.3], [-0.2], [0.7]])

    def force(Ph, Dh):
        a = Ph[0, 0] / psi1[0, 0]
        return (a * psi1) / Dh ** 2

    Psi, V = g.D(cfg.a_ini) * psi1, psi1.copy()
    for row in tab:
        Psi, V = nbody.step(cfg, Psi, V, row, None, force_fn=force)
        np.testing.assert_allclose(V, psi1, rtol=1e-12)
        np.testing.assert_allclose(Psi, row[6] * psi1, rtol=1e-12)


@pytest.mark.parametrize("time_var", ["D", "a"])
def test_bullfrog_2lpt_consistency_mock_force(time_var):
    # Sec. 2.4: BullFrog's alpha makes the velocity after each step equal the
    # 2LPT velocity psi1 + E'(D_{n+1}) psi2 when the force is the 2LPT force.
    # At a particle displaced by a psi1 + b psi2 the second-order force is
    # g = a psi1 + (b - a^2) psi2 (from d^2x/dD^2 = (3 gamma / D'^2)(g - D dx/dD)
    # and the E equation); FastPM (1LPT-consistent only) must not satisfy it.
    om = 0.3
    cfg = nbody.Config(n_part=1, n_mesh=1, box=1.0, omega_m=om, a_ini=0.02, a_end=1.0,
                       n_steps=6, time_var=time_var)
    g = cfg.get_growth()
    psi1 = np.array([[0.8], [0.0], [0.0]])
    psi2 = np.array([[0.0], [1.3], [0.0]])

    def force(Ph, Dh):
        a = Ph[0, 0] / psi1[0, 0]
        b = Ph[1, 0] / psi2[1, 0]
        return (a * psi1 + (b - a * a) * psi2) / Dh ** 2

    for stepper, ok in (("bullfrog", True), ("fastpm", False)):
        tab = cosmology.step_table(g, cfg.a_ini, cfg.a_end, cfg.n_steps, stepper, time_var)
        errs = []
        for row in tab:
            # one step from the exact 2LPT state at D_n
            a0 = g.a_of_D(row[5])
            Psi = g.D(a0) * psi1 + g.E(a0) * psi2
            V = psi1 + g.dE_dD(a0) * psi2
            Psi, V = nbody.step(cfg, Psi, V, row, None, force_fn=force)
            a1 = g.a_of_D(row[6])
            expect = psi1 + g.dE_dD(a1) * psi2
            errs.append(np.max(np.abs(V - expect)) / np.max(np.abs(expect)))
        if ok:
            assert max(errs) < 1e-9, errs
        else:
            assert max(errs) > 1e-3, errs


def test_bbks_limits():
    om, h = 0.3, 0.7
    # T -> 1 on large scales
    assert cosmology.bbks_transfer(1e-6, om, h) == pytest.approx(1.0, rel=1e-4)
    # small scales: T -> ln(2.34 q) / (2.34 q) * (6.71 q)^-1
    q = 1e5
    k = q * om * h
    asym = math.log(2.34 * q) / (2.34 * q) / (6.71 * q)
    assert cosmology.bbks_transfer(k, om, h) == pytest.approx(asym, rel=2e-3)


def test_sigma8_normalisation_independent_quadrature():
    pk = cosmology.LinearSpectrum(0.3, 0.7, 0.96, 0.8)
    # recompute sigma8 with a plain trapezoid on a dense log grid (not quad)
    lnk = np.linspace(math.log(1e-6), math.log(1e3), 400001)
    k = np.exp(lnk)
    x = 8.0 * k
    W = 3 * (np.sin(x) - x * np.cos(x)) / x ** 3
    W[x < 1e-3] = 1 - x[x < 1e-3] ** 2 / 10
    f = k ** 3 * pk(k) * W ** 2 / (2 * math.pi ** 2)
    s2 = np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(lnk))
    assert math.sqrt(s2) == pytest.approx(0.8, rel=1e-6)
    # P scales as sigma8^2
    pk2 = cosmology.LinearSpectrum(0.3, 0.7, 0.96, 1.6)
    assert pk2(0.1) == pytest.approx(4 * pk(0.1), rel=1e-9)


def test_table4_defaults_in_config():
    c = _paper_constants()
    cfg = nbody.Config(n_part=8, n_mesh=8, box=1.0)
    assert cfg.grad_order == c["default_grad_order"]
    assert cfg.lap_order == c["default_lap_order"]
    assert cfg.order == c["default_worder"]
