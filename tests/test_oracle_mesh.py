"""Pins of the oracle's mesh operations (Table 1, Table 2, Sec. 2.5, App. C)
against brute force, closed forms and invariants."""
import math
from pathlib import Path

import numpy as np
import pytest
from scipy import integrate, special

from oracle import mesh, nbody

GOLDEN = Path(__file__).parent / "golden"


def _stencils():
    rows = []
    for line in (GOLDEN / "table2_stencils.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            parts = line.split()
            rows.append((parts[0], int(parts[1]), float(parts[2]), [float(c) for c in parts[3:]]))
    return rows


@pytest.mark.parametrize("order", [2, 3, 4])
def test_kernel_partition_of_unity_and_first_moment(order):
    rng = np.random.default_rng(0)
    for x in rng.uniform(-3, 3, 50):
        m = np.arange(-6, 7)
        w = mesh.kernel_W(order, x - m)
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        assert (m * w).sum() == pytest.approx(x, abs=1e-13)


@pytest.mark.parametrize("order,p", [(2, 2), (3, 3), (4, 4)])
def test_kernel_fourier_transform_table1(order, p):
    # Table 1: W^(k) = sinc^p(k/2) with k in units of k_Ny and sinc(x) = sin(pi x)/(pi x);
    # with x in cells, k_Ny = pi, so W^(k) = [sin(k/2) / (k/2)]^p for k in rad/cell.
    for k in (0.3, 1.0, 2.0, 3.0):
        val, _ = integrate.quad(lambda x: mesh.kernel_W(order, x) * math.cos(k * x), -2.5, 2.5,
                                points=[-2, -1.5, -1, -0.5, 0, 0.5, 1, 1.5, 2], limit=200,
                                epsabs=1e-15, epsrel=1e-14)
        kt = k / math.pi
        assert val == pytest.approx(np.sinc(kt / 2.0) ** p, abs=1e-12)


@pytest.mark.parametrize("order", [2, 3])
def test_kernel_fourier_1d_is_the_aliased_deposit_spectrum(order):
    # Poisson summation: the DFT of one particle's deposit at sub-cell offset x0 is
    # sum_m W^(k + 2 pi m / H) exp(-i (k + 2 pi m / H) x0) (on the ky = kz = 0 line,
    # i.e. the deposit summed over y and z); averaged over 1024 evenly spaced offsets
    # the cross terms m != m' vanish unless m - m' is a multiple of 1024, so
    # E|rho^(k)|^2 = sum_m W^(k_m)^2 to ~1e-7 -- an independent check of Table 1's
    # W^ = sinc^p(k/2) (units, the pi in sinc, the power p)
    n, L = 16, 16.0
    H = L / n
    offs = (np.arange(1024) + 0.5) / 1024 * H
    acc = np.zeros(n)
    for x0 in offs:
        X = np.array([[3 * H + x0], [0.0], [0.0]])
        rho = mesh.scatter(X, None, n, L, order).sum(axis=(0, 1))
        acc += np.abs(np.fft.fft(rho)) ** 2
    acc /= len(offs)
    k = mesh.wavenumbers(n, L)
    ms = np.arange(-400, 401)
    expected = sum(mesh.kernel_fourier_1d(k + 2 * math.pi * m / H, H, order) ** 2 for m in ms)
    np.testing.assert_allclose(acc, expected, rtol=2e-6, atol=1e-12)


@pytest.mark.parametrize("order", [2, 3])
def test_deconvolved_force_multiplier(order):
    # deconvolution divides by the squared 3D kernel: ratio -> 1 as k -> 0, and on a
    # Nyquist plane of one axis the factor is (pi/2)^(2p) (Table 1: W^ = (2/pi)^p at kt = 1)
    n, L = 16, 40.0
    plain = mesh.force_multipliers(n, L, 4, 0)
    dec = mesh.force_multipliers(n, L, 4, 0, deconvolve_order=order)
    h = n // 2
    # x component at (kx, ky, kz) = (1, 0, 0): ratio 1 / sinc^(2p)(1/16) (close to 1)
    r1 = dec[0][0, 0, 1] / plain[0][0, 0, 1]
    assert 1.0 < r1 < 1.05
    np.testing.assert_allclose(r1, (math.sin(math.pi / 16) / (math.pi / 16)) ** (-2 * order), rtol=1e-12)
    # y component on the kx = Nyquist plane at ky = 1 (the x-gradient vanishes there)
    r2 = dec[1][0, 1, h] / plain[1][0, 1, h]
    np.testing.assert_allclose(r2, (math.pi / 2) ** (2 * order) * (math.sin(math.pi / 16) / (math.pi / 16)) ** (-2 * order),
                               rtol=1e-12)
    # k = 0 stays zero
    assert dec[0][0, 0, 0] == 0 and dec[2][0, 0, 0] == 0


@pytest.mark.parametrize("order", [2, 3, 4])
def test_kernel_derivative_matches_finite_difference(order):
    xs = np.array([-1.7, -1.2, -0.8, -0.3, 0.2, 0.6, 1.1, 1.6])
    side = np.sign(xs)
    eps = 1e-6
    fd = (mesh.kernel_W(order, xs + eps) - mesh.kernel_W(order, xs - eps)) / (2 * eps)
    np.testing.assert_allclose(mesh.kernel_dW(order, xs, side), fd, atol=1e-8)


@pytest.mark.parametrize("order,support", [(2, 8), (3, 27), (4, 64)])
def test_deposit_mass_conservation_and_support(order, support):
    rng = np.random.default_rng(1)
    n, L = 8, 10.0
    X = rng.uniform(0, L, (3, 200))
    rho = mesh.scatter(X, None, n, L, order)
    assert rho.sum() == pytest.approx(200.0, rel=1e-14)
    one = mesh.scatter(X[:, :1], None, n, L, order)
    assert np.count_nonzero(one > 1e-15) == support   # Table 1 discrete support


def test_deposit_unperturbed_lattice_is_uniform():
    for order in (2, 3, 4):
        for n in (8, 12):
            q = nbody.lattice(n, 5.0)
            d = mesh.density_contrast(q, n, 5.0, order)
            np.testing.assert_allclose(d, 0.0, atol=1e-13)


def test_cic_and_tsc_weights_by_hand():
    n, L = 16, 16.0   # H = 1
    X = np.array([[3.25], [4.5], [5.75]])
    rho = mesh.scatter(X, None, n, L, 2)
    # CIC: x: cells 3,4 weights .75,.25 ; y: 4,5 .5,.5 ; z: 5,6 .25,.75
    assert rho[5, 4, 3] == pytest.approx(0.25 * 0.5 * 0.75)
    assert rho[6, 5, 4] == pytest.approx(0.75 * 0.5 * 0.25)
    assert rho[6, 4, 3] == pytest.approx(0.75 * 0.5 * 0.75)
    # TSC: x = 3.25 -> nearest 3, d = .25 : (1/2)(1/4)^2, 3/4 - 1/16, (1/2)(3/4)^2
    rho3 = mesh.scatter(X, None, n, L, 3)
    wx = [0.5 * 0.25 ** 2, 0.75 - 0.0625, 0.5 * 0.75 ** 2]
    # y = 4.5 -> nearest 5 (ties up), d = -.5: (1/2)(1)^2, 3/4 - 1/4, 0
    wy = [0.5, 0.5, 0.0]
    # z = 5.75 -> nearest 6, d = -.25
    wz = [0.5 * 0.75 ** 2, 0.75 - 0.0625, 0.5 * 0.25 ** 2]
    for a in range(3):
        for b in range(3):
            for c in range(3):
                assert rho3[5 + a, 4 + b, 2 + c] == pytest.approx(wz[a] * wy[b] * wx[c], abs=1e-15)


def test_periodic_wrap():
    n, L = 8, 8.0
    X = np.array([[7.5], [0.0], [7.9]])
    rho = mesh.scatter(X, None, n, L, 2)
    # x = 7.5: cells 7, 0 (wrapped) with .5, .5; z = 7.9: cells 7 (.1) and 0 (.9)
    assert rho[7, 0, 7] == pytest.approx(0.1 * 1.0 * 0.5)
    assert rho[0, 0, 0] == pytest.approx(0.9 * 1.0 * 0.5)
    assert rho[0, 0, 7] == pytest.approx(0.9 * 1.0 * 0.5)
    assert rho.sum() == pytest.approx(1.0)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_scatter_gather_adjoint(order):
    # App. C: <scatter(w), rho> = <w, gather(rho)>
    rng = np.random.default_rng(2)
    n, L = 8, 3.0
    X = rng.uniform(-L, 2 * L, (3, 300))
    w = rng.normal(size=300)
    rho = rng.normal(size=(n, n, n))
    lhs = np.sum(mesh.scatter(X, w, n, L, order) * rho)
    rhs = np.sum(w * mesh.gather(rho, X, L, order))
    assert lhs == pytest.approx(rhs, rel=1e-13)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_gather_grad_matches_finite_difference(order):
    rng = np.random.default_rng(3)
    n, L = 8, 8.0
    X = rng.uniform(0, L, (3, 50))
    # keep CIC particles away from cell faces (kinks)
    X = np.floor(X) + rng.uniform(0.1, 0.9, X.shape)
    rho = rng.normal(size=(n, n, n))
    g = mesh.gather_grad(rho, X, L, order)
    eps = 1e-6
    for d in range(3):
        e = np.zeros_like(X)
        e[d] = eps
        fd = (mesh.gather(rho, X + e, L, order) - mesh.gather(rho, X - e, L, order)) / (2 * eps)
        np.testing.assert_allclose(g[d], fd, atol=1e-7)


def test_table2_fourier_kernels_are_stencil_transforms():
    # DFT of the printed stencils vs the Fourier kernels (with the order-2
    # Laplacian sign reading).  H = 0.7; k over the whole Brillouin zone.
    H = 0.7
    k = np.linspace(-math.pi / H, math.pi / H, 41)
    for kind, order, den, coef in _stencils():
        m = (len(coef) - 1) // 2
        offs = np.arange(-m, m + 1)
        # f'(x) ~ sum_m c_m f(x + m H) / H  ->  multiplier sum_m c_m e^{i k m H} / H
        p = 1 if kind == "gradient" else 2
        ft = np.array([np.sum(np.array(coef) / den * np.exp(1j * kk * offs * H)) for kk in k]) / H ** p
        mine = (mesh.grad_kernel_1d(k, H, order) if kind == "gradient"
                else mesh.laplace_kernel_1d(k, H, order))
        np.testing.assert_allclose(mine, ft, atol=1e-12 * (1 + np.max(np.abs(ft))))


def test_force_single_mode_exact_kernels():
    # delta = cos(k0.r): g = -grad Lap^-1 delta = -k0 sin(k0.r) / |k0|^2 (exact kernels).
    n, L = 16, 10.0
    H = L / n
    r = np.arange(n) * H
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    k0 = 2 * math.pi / L * np.array([2.0, -1.0, 3.0])
    phase = k0[0] * x + k0[1] * y + k0[2] * z
    delta = np.cos(phase)
    g = mesh.force_field(delta, L, grad_order=0, lap_order=0)
    for c in range(3):
        np.testing.assert_allclose(g[c], -k0[c] * np.sin(phase) / np.dot(k0, k0), atol=1e-12)


@pytest.mark.parametrize("grad_order", [2, 4, 6])
@pytest.mark.parametrize("lap_order", [0, 2, 4])
def test_fd_force_equals_real_space_stencil(grad_order, lap_order):
    # the Fourier gradient must act like the Table 2 stencil applied in real space
    rng = np.random.default_rng(4)
    n, L = 16, 5.0
    H = L / n
    delta = rng.normal(size=(n, n, n))
    delta -= delta.mean()
    ms_phi = mesh.force_multipliers(n, L, 0, lap_order)
    # potential phi = Lap^-1 delta (multiplier 1/K_lap): recover from the exact-gradient force
    k1 = mesh.wavenumbers(n, L)
    lap = sum(mesh.laplace_kernel_1d(kc, H, lap_order)
              for kc in np.meshgrid(k1, k1, k1, indexing="ij"))
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(lap != 0, 1 / lap, 0)
    inv[0, 0, 0] = 0
    phi = np.fft.ifftn(inv * np.fft.fftn(delta)).real
    st = {o: (d, c) for kind, o, d, c in _stencils() if kind == "gradient"}
    den, coef = st[grad_order]
    mm = (len(coef) - 1) // 2
    g = mesh.force_field(delta, L, grad_order, lap_order)
    axes = {0: 2, 1: 1, 2: 0}   # component x is array axis 2
    for c in range(3):
        d = np.zeros_like(phi)
        for o, cc in zip(range(-mm, mm + 1), coef):
            d += cc / den * np.roll(phi, -o, axis=axes[c])
        d /= H
        # the Nyquist plane of component c is zeroed in the Fourier kernel; the
        # stencil also annihilates it (sin(pi) = 0), so they agree everywhere
        np.testing.assert_allclose(g[c], -d, atol=1e-11)
    del ms_phi


@pytest.mark.parametrize("order", [2, 3])
def test_self_force_and_momentum_conservation(order):
    # matched deposit/interpolation with an odd gradient kernel: sum_i A_i = 0,
    # a lone particle feels no force, and a pair feels equal and opposite forces.
    rng = np.random.default_rng(5)
    cfg = nbody.Config(n_part=4, n_mesh=16, box=20.0, order=order)
    q = np.zeros((3, 1))
    A1 = nbody.accel(cfg, rng.uniform(0, 20, (3, 1)), q, 1.0)
    np.testing.assert_allclose(A1, 0.0, atol=1e-12)
    q2 = np.zeros((3, 2))
    A2 = nbody.accel(cfg, rng.uniform(0, 20, (3, 2)), q2, 1.0)
    np.testing.assert_allclose(A2[:, 0], -A2[:, 1], atol=1e-12)
    qn = np.zeros((3, 100))
    An = nbody.accel(cfg, rng.uniform(0, 20, (3, 100)), qn, 1.0)
    np.testing.assert_allclose(An.sum(axis=1), 0.0, atol=1e-10)


def _ewald_field(r, L, alpha=None, nreal=3, kmax=12):
    """Periodic 1/r^2 field E = sum_n r_n/|r_n|^3 (minus uniform background) by Ewald summation."""
    alpha = alpha or 5.0 / L
    E = np.zeros(3)
    rng_ = range(-nreal, nreal + 1)
    for i in rng_:
        for j in rng_:
            for k in rng_:
                rv = r + L * np.array([i, j, k])
                d = np.linalg.norm(rv)
                E += rv / d ** 3 * (special.erfc(alpha * d)
                                    + 2 * alpha * d / math.sqrt(math.pi) * math.exp(-(alpha * d) ** 2))
    for i in range(-kmax, kmax + 1):
        for j in range(-kmax, kmax + 1):
            for k in range(-kmax, kmax + 1):
                if i == j == k == 0:
                    continue
                kv = 2 * math.pi / L * np.array([i, j, k])
                k2 = kv @ kv
                E += 4 * math.pi / L ** 3 * kv / k2 * math.exp(-k2 / (4 * alpha ** 2)) * math.sin(kv @ r)
    return E


def test_pair_force_is_newtonian_at_large_separation():
    # g = -grad Lap^-1 delta, delta = (M/N) rho - 1: a particle is a point source
    # of strength L^3/N, so the field of particle 2 at particle 1 is
    # -(L^3/N)/(4 pi) E_periodic(X1 - X2).  Default kernels (Table 4: 4th-order
    # gradient, exact Laplacian), CIC.  (With the exact ik gradient the PM pair
    # force rings around the Newtonian value, which is why the paper prefers
    # finite-difference gradients, App. A.4.)
    n, L = 32, 32.0
    cfg = nbody.Config(n_part=2, n_mesh=n, box=L, order=2, grad_order=4, lap_order=0)
    for sep in (6.0, 9.0, 12.0):
        X = np.array([[10.3, 10.3 + sep], [11.6, 11.6], [9.2, 9.2]])
        A = nbody.accel(cfg, X, np.zeros_like(X), 1.0)
        expect = -(L ** 3 / 2) / (4 * math.pi) * _ewald_field(X[:, 0] - X[:, 1], L)
        err = np.linalg.norm(A[:, 0] - expect) / np.linalg.norm(expect)
        assert err < 0.01, (sep, A[:, 0], expect)


def test_power_spectrum_plane_wave_closed_form():
    # delta = A cos(k_F x): bin 0 ([k_F/2, 3k_F/2)) holds the 6 modes |m| = 1 and
    # the 12 modes |m| = sqrt 2; two of them have |delta^|^2 = (A M / 2)^2, so
    # P = (L^3/M^2) * 2 (A M/2)^2 / 18 = L^3 A^2 / 36.
    n, L, Amp = 16, 7.0, 0.3
    r = np.arange(n) * L / n
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    delta = Amp * np.cos(2 * math.pi / L * x)
    k, P, cnt = mesh.power_spectrum(delta, L, 8)
    assert cnt[0] == 18
    assert P[0] == pytest.approx(L ** 3 * Amp ** 2 / 36, rel=1e-12)
    assert k[0] == pytest.approx(2 * math.pi / L * (6 + 12 * math.sqrt(2)) / 18, rel=1e-12)
    np.testing.assert_allclose(P[1:], 0.0, atol=1e-20)
    # mode counts: every mode of the grid with 1/2 <= |m| < n_bins + 1/2 is counted once
    m = np.fft.fftfreq(n, 1.0 / n)
    mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
    mm = np.sqrt(mx ** 2 + my ** 2 + mz ** 2)
    assert cnt.sum() == np.count_nonzero((mm >= 0.5) & (mm < 8.5))


def test_power_spectrum_white_noise_is_flat():
    rng = np.random.default_rng(6)
    n, L = 32, 100.0
    delta = rng.normal(size=(n, n, n))
    k, P, cnt = mesh.power_spectrum(delta, L, 15)
    expect = L ** 3 / n ** 3      # <|delta^|^2> = M sigma^2
    ok = cnt > 200
    rel = np.abs(P[ok] / expect - 1)
    assert np.all(rel < 5 / np.sqrt(cnt[ok] / 2))
