"""Pins of the oracle's N-body layer: Zel'dovich ICs (Sec. 2.2), the full PM
stepper (Eq. dkd) on an exactly solvable plane wave, and the adjoint method
(Sec. 2.7, Table 5, App. C) against central finite differences."""
import math

import numpy as np
import pytest

from oracle import cosmology, mesh, nbody


def _noise(n, seed):
    return np.random.default_rng(seed).standard_normal((n, n, n))


def test_ic_linear_density_response_and_sign():
    # Displace the lattice by a tiny D psi1 and deposit with TSC: to first order
    # (W(0) = 3/4, W(+-1) = 1/8, W'(+-1) = -+1/2 from Table 1) the deposit is
    # -sum_c [central difference along c] [1/8 3/4 1/8 smoothing across c] of u_c,
    # so delta_dep^(k) = -i D sum_c sin(k_c H)/H prod_{d != c} s(k_d) psi1_c^(k),
    # s(k) = 3/4 + cos(k H)/4.
    # (a) on the axis modes the ratio delta_dep^ / w^ is real and positive (sign of
    #     psi1 = i k / k^2 delta / D(1) and no conjugation);
    # (b) the deposited power, corrected by the difference operator, is the linear
    #     spectrum times (D / D(1))^2 within cosmic variance.
    n, L = 32, 256.0
    cfg = nbody.Config(n_part=n, n_mesh=n, box=L, order=3)
    w = _noise(n, 11)
    g = cfg.get_growth()
    _, psi1 = nbody.zeldovich_ic(cfg, w)
    D = 1e-5 / np.sqrt(np.mean(psi1 ** 2)) * (L / n)   # rms displacement 1e-5 cells
    X = nbody.lattice(n, L) + D * psi1
    dep = np.fft.fftn(mesh.density_contrast(X, n, L, order=3))
    wk = np.fft.fftn(w)
    for m in (1, 2, 3):
        for idx in ((0, 0, m), (0, m, 0), (m, 0, 0)):
            r = dep[idx] / wk[idx]
            assert abs(r.imag) < 1e-3 * abs(r.real)
            assert r.real > 0
    H = L / n
    k1 = mesh.wavenumbers(n, L)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        s = [0.75 + 0.25 * np.cos(kc * H) for kc in (kx, ky, kz)]
        op = (np.sin(kx * H) * kx * s[1] * s[2] + np.sin(ky * H) * ky * s[0] * s[2]
              + np.sin(kz * H) * kz * s[0] * s[1]) / H / k2
    op[0, 0, 0] = 1.0
    corrected = np.fft.ifftn(dep / op).real * g.D(1.0) / D
    k, P, cnt = mesh.power_spectrum(corrected, L, 12)
    pk = cosmology.LinearSpectrum(cfg.omega_m, cfg.h, cfg.n_s, cfg.sigma8)
    # bins well inside the Nyquist sphere; mean P over a bin vs P at the bin's k
    # (the spectrum varies across a bin; allow 4 sigma of cosmic variance + 5%)
    for b in range(2, 12):
        sig = math.sqrt(2.0 / cnt[b])
        assert abs(P[b] / pk(k[b]) - 1) < 4 * sig + 0.05, (b, P[b], pk(k[b]))


def test_ic_zero_modes():
    n, L = 16, 100.0
    cfg = nbody.Config(n_part=n, n_mesh=n, box=L)
    Psi, V = nbody.zeldovich_ic(cfg, _noise(n, 3))
    for c in range(3):
        f = np.fft.fftn(V[c].reshape(n, n, n))
        assert abs(f[0, 0, 0]) < 1e-10
        assert np.max(np.abs(f[n // 2, :, :])) < 1e-10
        assert np.max(np.abs(f[:, :, n // 2])) < 1e-10
        m = np.fft.fftfreq(n, 1 / n)
        mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
        assert np.max(np.abs(f[np.sqrt(mx ** 2 + my ** 2 + mz ** 2) > n / 2])) < 1e-10
    np.testing.assert_allclose(Psi, cfg.get_growth().D(cfg.a_ini) * V, rtol=1e-15)


def _lattice_fields(n, L):
    q = np.arange(n) * (L / n)
    qz, qy, qx = np.meshgrid(q, q, q, indexing="ij")
    return qx, qy, qz


def test_lpt2_vanishes_for_a_planar_wave():
    # planar symmetry: psi_i,j is non-zero for i = j = x only, so mu_2L = 0 and psi^(2) = 0
    n, L = 16, 100.0
    qx, qy, qz = _lattice_fields(n, L)
    k = 2 * math.pi * 2 / L
    psi1 = np.stack([(3.0 * np.sin(k * qx)).reshape(-1), np.zeros(n ** 3), np.zeros(n ** 3)])
    assert np.max(np.abs(nbody.lpt2_term(psi1, L))) < 1e-12


def test_lpt2_crossed_waves_closed_form():
    # psi1 = (A sin kx, B sin ky, 0): mu_2L = psi_x,x psi_y,y = A B k^2 cos kx cos ky,
    # L2 = -(3/7) mu_2L, Lap^-1 L2 = (3/14) A B cos kx cos ky (|k|^2 = 2 k^2), so
    # psi^(2) = grad of that = (3/14) A B k (-sin kx cos ky, -cos kx sin ky, 0)
    n, L = 16, 100.0
    qx, qy, qz = _lattice_fields(n, L)
    k = 2 * math.pi * 3 / L
    A, B = 2.0, -1.5
    psi1 = np.stack([(A * np.sin(k * qx)).reshape(-1), (B * np.sin(k * qy)).reshape(-1), np.zeros(n ** 3)])
    psi2 = nbody.lpt2_term(psi1, L)
    c = 3.0 / 14.0 * A * B * k
    np.testing.assert_allclose(psi2[0], (-c * np.sin(k * qx) * np.cos(k * qy)).reshape(-1), atol=1e-12)
    np.testing.assert_allclose(psi2[1], (-c * np.cos(k * qx) * np.sin(k * qy)).reshape(-1), atol=1e-12)
    assert np.max(np.abs(psi2[2])) < 1e-12


def test_lpt2_ic_state():
    # Psi0 = D psi1 + D^2 psi2 and V0 = psi1 + 2 D psi2 (the D-derivative of Psi)
    cfg1 = nbody.Config(n_part=16, n_mesh=16, box=100.0)
    cfg2 = nbody.Config(n_part=16, n_mesh=16, box=100.0, lpt_order=2)
    w = np.random.default_rng(3).standard_normal((16, 16, 16))
    P1, V1 = nbody.zeldovich_ic(cfg1, w)
    P2, V2 = nbody.zeldovich_ic(cfg2, w)
    D = cfg1.get_growth().D(cfg1.a_ini)
    psi2 = nbody.lpt2_term(V1, 100.0)
    np.testing.assert_allclose(P2, P1 + D ** 2 * psi2, atol=1e-14)
    np.testing.assert_allclose(V2, V1 + 2 * D * psi2, atol=1e-14)
    # second order is small at a = 0.02 but not zero
    assert 0 < np.max(np.abs(P2 - P1)) < 1e-2 * np.max(np.abs(P1))


def test_plane_wave_follows_zeldovich_solution():
    # A planar wave psi1 = A sin(2 pi q_x / L) e_x stays exactly Zel'dovich
    # (X = q + D psi1) until shell crossing; the PM run must follow it up to
    # force-resolution error.  Shell crossing at D A k = 1: pick D(1) A k = 0.5.
    # TSC: with CIC a lattice sits on the kinks of W, so the linear density
    # response is a one-sided difference whose sign flips with the sign of the
    # displacement (O(kH) harmonics, ~10% here); TSC is smooth at the nodes.
    n, L = 32, 256.0
    cfg = nbody.Config(n_part=n, n_mesh=n, box=L, order=3, n_steps=6)
    g = cfg.get_growth()
    kw = 2 * math.pi / L
    Amp = 0.5 / (g.D(1.0) * kw)
    q = nbody.lattice(n, L)
    psi1 = np.zeros_like(q)
    psi1[0] = Amp * np.sin(kw * q[0])
    Psi, V = nbody.run(cfg, g.D(cfg.a_ini) * psi1, psi1.copy())
    expect = g.D(1.0) * psi1
    err = np.max(np.abs(Psi - expect)) / np.max(np.abs(expect))
    assert err < 0.025, err
    np.testing.assert_allclose(Psi[1:], 0.0, atol=1e-9 * Amp)
    # the residual is force resolution: a finer mesh halves it
    cfg2 = nbody.Config(n_part=n, n_mesh=2 * n, box=L, order=3, n_steps=6)
    Psi2, _ = nbody.run(cfg2, g.D(cfg.a_ini) * psi1, psi1.copy())
    assert np.max(np.abs(Psi2 - expect)) / np.max(np.abs(expect)) < 0.75 * err
    # and the wrong sign of the force would push particles the other way
    assert np.sum((Psi[0] - g.D(cfg.a_ini) * psi1[0]) * psi1[0]) > 0


def _small_cfg(order, **kw):
    base = dict(n_part=8, n_mesh=8, box=40.0, order=order, n_steps=3, a_ini=0.05, sigma8=2.5)
    base.update(kw)
    return nbody.Config(**base)


@pytest.mark.parametrize("order", [3, 2])
def test_accel_vjp_matches_finite_difference(order):
    rng = np.random.default_rng(7)
    cfg = _small_cfg(order)
    q = nbody.lattice(8, 40.0)
    Psi = rng.normal(scale=3.0, size=q.shape)
    u = rng.normal(size=q.shape)
    e = rng.normal(size=q.shape)
    Dh = 0.4
    vjp = nbody.accel_vjp(cfg, Psi, q, Dh, u)
    eps = 1e-6
    fd = np.sum(u * (nbody.accel(cfg, Psi + eps * e, q, Dh) - nbody.accel(cfg, Psi - eps * e, q, Dh))) / (2 * eps)
    tol = 1e-6 if order == 3 else 1e-4
    assert np.sum(vjp * e) == pytest.approx(fd, rel=tol)


def _loss_pipeline(cfg, w, target, sigma=0.1):
    Psi0, V0 = nbody.zeldovich_ic(cfg, w)
    Psi, V = nbody.run(cfg, Psi0, V0)
    X = np.mod(nbody.lattice(cfg.n_part, cfg.box) + Psi, cfg.box)
    delta = mesh.density_contrast(X, cfg.n_mesh, cfg.box, cfg.order)
    return 0.5 * np.sum(((delta - target) / sigma) ** 2), Psi, V, delta


@pytest.mark.parametrize("order", [3, 2])
def test_adjoint_gradient_matches_finite_difference(order):
    cfg = _small_cfg(order)
    n = cfg.n_part
    w = _noise(n, 21)
    target = 0.3 * _noise(n, 22)
    sigma = 0.1
    Lval, Psi, V, delta = _loss_pipeline(cfg, w, target, sigma)
    Xa = nbody.density_vjp(cfg, Psi, (delta - target) / sigma ** 2)
    Psi0, V0, Xa0, Va0 = nbody.adjoint(cfg, Psi, V, Xa, np.zeros_like(V))
    # reversibility of the backward primal (Sec. 2.7)
    Pi, Vi = nbody.zeldovich_ic(cfg, w)
    np.testing.assert_allclose(Psi0, Pi, atol=1e-10 * np.max(np.abs(Pi)))
    np.testing.assert_allclose(V0, Vi, atol=1e-10 * np.max(np.abs(Vi)))
    wa, ds8 = nbody.ic_vjp(cfg, Xa0, Va0, w)
    rng = np.random.default_rng(23)
    eps = 1e-5
    tol = 2e-6 if order == 3 else 5e-4
    for _ in range(4):
        e = rng.normal(size=w.shape)
        lp = _loss_pipeline(cfg, w + eps * e, target, sigma)[0]
        lm = _loss_pipeline(cfg, w - eps * e, target, sigma)[0]
        assert np.sum(wa * e) == pytest.approx((lp - lm) / (2 * eps), rel=tol)
    s8 = cfg.sigma8
    c_p = _small_cfg(order, sigma8=s8 * (1 + 1e-6))
    c_m = _small_cfg(order, sigma8=s8 * (1 - 1e-6))
    fd = (_loss_pipeline(c_p, w, target, sigma)[0] - _loss_pipeline(c_m, w, target, sigma)[0]) / (2e-6 * s8)
    assert ds8 == pytest.approx(fd, rel=tol)


def test_spectral_operator_transpose_is_conjugate_multiplier():
    # <F_c x, y> = <x, F_c^T y> with F_c^T the multiplier conj(m_c)  (App. C pullbacks)
    rng = np.random.default_rng(9)
    n, L = 8, 10.0
    ms = mesh.force_multipliers(n, L, 4, 2)
    x, y = rng.normal(size=(2, n, n, n))
    for m in ms:
        lhs = np.sum(mesh.apply_multiplier(x, m) * y)
        rhs = np.sum(x * mesh.apply_multiplier(y, np.conj(m)))
        assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.slow
def test_interlaced_force_is_closer_to_newtonian():
    # Interlacing (Sec. 2.8) reduces aliasing: the pair force of two particles
    # averaged over sub-cell offsets scatters less around its mean with two grids.
    n, L = 16, 16.0
    rng = np.random.default_rng(10)
    res = {}
    for inter in (False, True):
        cfg = nbody.Config(n_part=2, n_mesh=n, box=L, order=2, interlace=inter)
        vals = []
        for _ in range(12):
            p = rng.uniform(0, L, 3)
            d = np.array([3.0, 0.0, 0.0])
            X = np.stack([p, p + d], axis=1)
            A = nbody.accel(cfg, X, np.zeros_like(X), 1.0)
            vals.append(A[0, 0])
            np.testing.assert_allclose(A[:, 0], -A[:, 1], atol=1e-10)
        res[inter] = np.std(vals) / abs(np.mean(vals))
    assert res[True] < res[False]


# ---------------------------------------------------------------- forward mode (JVPs)

@pytest.mark.parametrize("order", [3, 4])
def test_scatter_dot_grad_is_the_scatter_tangent(order):
    # central differences of the (smooth-kernel) scatter along T, and the exact
    # transpose identity <scatter_dot_grad(T), m> = sum_i T_i . gather_grad(m)_i
    n, L = 8, 8.0
    rng = np.random.default_rng(21)
    X = rng.uniform(0, L, size=(3, 40))
    T = rng.normal(size=(3, 40))
    eps = 1e-6
    fd = (mesh.scatter(X + eps * T, None, n, L, order) - mesh.scatter(X - eps * T, None, n, L, order)) / (2 * eps)
    jv = mesh.scatter_dot_grad(X, T, n, L, order)
    assert np.max(np.abs(jv - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))
    m = rng.normal(size=(n, n, n))
    lhs = np.sum(jv * m)
    rhs = np.sum(T * mesh.gather_grad(m, X, L, order))
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


def test_accel_jvp_dot_product_with_vjp_and_finite_differences():
    n, L = 16, 100.0
    cfg = nbody.Config(n_part=n, n_mesh=n, box=L, order=3)
    rng = np.random.default_rng(22)
    q = nbody.lattice(n, L)
    P = rng.normal(scale=2.0, size=(3, n ** 3))
    T = rng.normal(size=(3, n ** 3))
    u = rng.normal(size=(3, n ** 3))
    Dh = 0.4
    jt = nbody.accel_jvp(cfg, P, q, Dh, T)
    vu = nbody.accel_vjp(cfg, P, q, Dh, u)
    assert np.sum(u * jt) == pytest.approx(np.sum(vu * T), rel=1e-10)
    eps = 1e-4
    fd = (nbody.accel(cfg, P + eps * T, q, Dh) - nbody.accel(cfg, P - eps * T, q, Dh)) / (2 * eps)
    assert np.max(np.abs(jt - fd)) < 1e-5 * np.max(np.abs(fd))


def test_run_jvp_matches_finite_differences():
    n, L = 16, 128.0
    cfg = nbody.Config(n_part=n, n_mesh=n, box=L, order=3, n_steps=3)
    w = np.random.default_rng(23).standard_normal((n, n, n))
    wt = np.random.default_rng(24).standard_normal((n, n, n))
    P0, V0 = nbody.zeldovich_ic(cfg, w)
    Pt0, Vt0 = nbody.zeldovich_ic(cfg, wt)          # the ICs are linear in the noise
    P, V, Pt, Vt = nbody.run_jvp(cfg, P0, V0, Pt0, Vt0)
    eps = 1e-5
    Pp, Vp = nbody.run(cfg, *nbody.zeldovich_ic(cfg, w + eps * wt))
    Pm, Vm = nbody.run(cfg, *nbody.zeldovich_ic(cfg, w - eps * wt))
    np.testing.assert_allclose(Pt, (Pp - Pm) / (2 * eps), atol=1e-6 * np.max(np.abs(Pt)))
    np.testing.assert_allclose(Vt, (Vp - Vm) / (2 * eps), atol=1e-6 * np.max(np.abs(Vt)))
    ref_P, _ = nbody.run(cfg, P0, V0)
    np.testing.assert_allclose(P, ref_P, atol=1e-12)


def test_power_spectrum_jvp_matches_finite_differences():
    n, L = 16, 100.0
    rng = np.random.default_rng(25)
    P = rng.normal(scale=3.0, size=(3, n ** 3))
    T = rng.normal(size=(3, n ** 3))
    k, dpk, cnt = nbody.power_spectrum_jvp(P, T, n, L, 8, order=3)
    eps = 1e-5
    X = nbody.lattice(n, L)

    def pk(Q):
        return mesh.power_spectrum(mesh.density_contrast(np.mod(X + Q, L), n, L, 3), L, 8)[1]

    fd = (pk(P + eps * T) - pk(P - eps * T)) / (2 * eps)
    np.testing.assert_allclose(dpk, fd, rtol=1e-6, atol=1e-9 * np.max(np.abs(fd)))


# ---------------------------------------------------------------- NUFFT force (exact band DFT)

def test_nufft_band_force_conserves_momentum_and_matches_pm_on_band_limited_density():
    n, L = 8, 40.0
    rng = np.random.default_rng(31)
    X = rng.uniform(0, L, size=(3, 300))
    A = nbody.nufft_band_force(X, n, L)
    # odd imaginary multiplier and |delta^|^2 even: the total force vanishes
    assert np.max(np.abs(A.sum(axis=1))) < 1e-10 * np.max(np.abs(A))
    # particles on the lattice, displaced along x by a single band mode: delta is then
    # band-limited to first order and the force equals the exact-kernel PM force at
    # the lattice points to second order in the amplitude
    n = 16
    q = nbody.lattice(n, L)
    eps, kk = 1e-4, 2 * math.pi * 3 / L
    Psi = np.zeros_like(q)
    Psi[0] = eps * np.sin(kk * q[0])
    A = nbody.nufft_band_force(q + Psi, n, L)
    # linear theory: delta = -div Psi = -eps k cos(k x), g = -grad Lap^-1 delta = +eps sin(k x)
    # (x only): the force is the displacement, as Zel'dovich consistency requires
    np.testing.assert_allclose(A[0], eps * np.sin(kk * q[0]), atol=1e-3 * eps)
    assert np.max(np.abs(A[1:])) < 1e-3 * eps


def test_es_nufft_approximates_the_band_dft():
    # the NUFFT algorithm (ES kernel, width 5, beta = 2.3 w, grid upsampled twice,
    # deconvolution by the kernel's continuous transform both ways) against the
    # exact band DFT: error ~1e-4 of the force, the 10^-(w-1) accuracy expected of a
    # width-5 ES kernel at upsampling 2
    n, L = 8, 40.0
    X = np.random.default_rng(32).uniform(0, L, size=(3, 400))
    out = mesh.nufft_force(X, n, L)
    ref = nbody.nufft_band_force(X, n, L)
    assert np.max(np.abs(out - ref)) < 2e-4 * np.max(np.abs(ref))
    # a denser, smoother (lattice + small displacement) distribution: closer still
    n = 16
    q = nbody.lattice(n, L)
    X = np.mod(q + np.random.default_rng(33).normal(scale=0.5, size=q.shape), L)
    out = mesh.nufft_force(X, n, L)
    ref = nbody.nufft_band_force(X, n, L)
    assert np.max(np.abs(out - ref)) < 2e-4 * np.max(np.abs(ref))


def test_es_fourier_matches_discrete_sum():
    # the continuous transform of the ES kernel: a fine Riemann sum agrees
    nf = 32
    ph = mesh.es_fourier(nf)
    t = np.linspace(-2.5, 2.5, 200001)
    for m in (0, 3, 8, 15):
        val = np.trapezoid(mesh.es_kernel(t) * np.cos(2 * np.pi * m / nf * t), t)
        assert ph[m] == pytest.approx(val, rel=1e-8)
