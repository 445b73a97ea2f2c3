"""Oracle mesh operations: mass assignment, scatter/gather, Poisson force, P(k).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Layout conventions (shared with the inputs, not with any GPU code):
* a mesh with n cells per side is a float64 array of shape (n, n, n) indexed
  [z, y, x]; node j has position r_j = j H, H = L / n (reading: the paper does
  not say where mesh nodes sit; with nodes at j H an unperturbed particle
  lattice at q = i L / n_p deposits an exactly uniform density when n = n_p).
* particle positions are arrays of shape (3, N) with component 0 = x.
"""
import math

import numpy as np

ORDER_NAMES = {2: "CIC", 3: "TSC", 4: "PCS"}


# --------------------------------------------------------------------------
# 1D mass-assignment kernels, Table 1 (x in cells)
# --------------------------------------------------------------------------

def kernel_W(order, x):
    """W(x) of Table 1: CIC (order 2), TSC (3), PCS (4)."""
    ax = np.abs(np.asarray(x, dtype=np.float64))
    if order == 2:
        return np.where(ax <= 1.0, 1.0 - ax, 0.0)
    if order == 3:
        return np.where(ax <= 0.5, 0.75 - ax ** 2,
                        np.where(ax <= 1.5, 0.5 * (1.5 - ax) ** 2, 0.0))
    if order == 4:
        return np.where(ax <= 1.0, (4.0 - 6.0 * ax ** 2 + 3.0 * ax ** 3) / 6.0,
                        np.where(ax <= 2.0, (2.0 - ax) ** 3 / 6.0, 0.0))
    raise ValueError(order)


def kernel_dW(order, x, side):
    """dW/dx of Table 1's kernels.

    At the kinks of CIC (x = 0) the derivative is not defined; ``side`` (an
    array of +1/-1, the sign of x that the tap was chosen on) selects the
    one-sided value that differentiating the forward assignment gives (the
    reading for tie-breaks: CIC cells are chosen by floor).
    """
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    s = np.where(x != 0.0, np.sign(x), side)
    if order == 2:
        return np.where(ax <= 1.0, -s, 0.0)
    if order == 3:
        return np.where(ax <= 0.5, -2.0 * x,
                        np.where(ax <= 1.5, -s * (1.5 - ax), 0.0))
    if order == 4:
        return np.where(ax <= 1.0, s * (-12.0 * ax + 9.0 * ax ** 2) / 6.0,
                        np.where(ax <= 2.0, -s * 0.5 * (2.0 - ax) ** 2, 0.0))
    raise ValueError(order)


def taps_1d(order, u):
    """Cells touched by a particle at u (in cells) and their signed offsets.

    CIC: floor(u), floor(u)+1.  TSC: nearest node i0 = floor(u + 1/2) (ties
    rounded up) and its two neighbours.  PCS: floor(u)-1 .. floor(u)+2.
    Returns (list of integer cell arrays, list of x = j - u arrays, list of
    side arrays used for the one-sided derivative at a kink).
    """
    u = np.asarray(u, dtype=np.float64)
    if order == 2:
        i0 = np.floor(u)
        offs = [0, 1]
    elif order == 3:
        i0 = np.floor(u + 0.5)
        offs = [-1, 0, 1]
    elif order == 4:
        i0 = np.floor(u)
        offs = [-1, 0, 1, 2]
    else:
        raise ValueError(order)
    cells, xs, sides = [], [], []
    for o in offs:
        j = i0 + o
        cells.append(j.astype(np.int64))
        xs.append(j - u)
        # a tap at or left of u was chosen as "x <= 0"; right of it as "x > 0"
        sides.append(np.where(o <= 0, -1.0, 1.0) * np.ones_like(u))
    return cells, xs, sides


def _tap_products(X, n, L, order, shift=0.0):
    """For every particle and every 3D tap: flat mesh index, weight, and the
    three derivative factors dW/dX_d (per unit length).  Brute-force product
    over the 1D taps (Table 1: the 3D kernel is the product of 1D kernels)."""
    H = L / n
    per_axis = []
    for d in range(3):
        u = np.mod(X[d] + shift, L) / H
        cells, xs, sides = taps_1d(order, u)
        w = [kernel_W(order, x) for x in xs]
        # d/dX of W(r_j - X) = -W'(j - u) / H
        dw = [-kernel_dW(order, x, s) / H for x, s in zip(xs, sides)]
        per_axis.append((cells, w, dw))
    out = []
    cz, wz, dz = per_axis[2]
    cy, wy, dy = per_axis[1]
    cx, wx, dx = per_axis[0]
    for a in range(len(cz)):
        for b in range(len(cy)):
            for c in range(len(cx)):
                idx = ((np.mod(cz[a], n) * n + np.mod(cy[b], n)) * n + np.mod(cx[c], n))
                weight = wz[a] * wy[b] * wx[c]
                grad = (dx[c] * wy[b] * wz[a], wx[c] * dy[b] * wz[a], wx[c] * wy[b] * dz[a])
                out.append((idx, weight, grad))
    return out


def scatter(X, weights, n, L, order, shift=0.0):
    """rho_j = sum_i w_i W(r_j - X_i - shift)  (App. C, scatter)."""
    M = n ** 3
    rho = np.zeros(M)
    w = np.ones(X.shape[1]) if weights is None else np.asarray(weights, dtype=np.float64)
    for idx, weight, _ in _tap_products(X, n, L, order, shift):
        rho += np.bincount(idx, weights=w * weight, minlength=M)
    return rho.reshape(n, n, n)


def gather(mesh, X, L, order, shift=0.0):
    """v_i = sum_j rho_j W(r_j - X_i - shift)  (App. C, gather)."""
    n = mesh.shape[0]
    flat = mesh.reshape(-1)
    v = np.zeros(X.shape[1])
    for idx, weight, _ in _tap_products(X, n, L, order, shift):
        v += flat[idx] * weight
    return v


def gather_grad(mesh, X, L, order, shift=0.0):
    """d/dX_i of gather: sum_j rho_j d/dX_i W(r_j - X_i)  -> array (3, N) (App. C)."""
    n = mesh.shape[0]
    flat = mesh.reshape(-1)
    g = np.zeros((3, X.shape[1]))
    for idx, _, grad in _tap_products(X, n, L, order, shift):
        for d in range(3):
            g[d] += flat[idx] * grad[d]
    return g


def scatter_dot_grad(X, T, n, L, order, shift=0.0):
    """Tangent of scatter(X, 1) along position tangents T (3, N):
    rho'_j = sum_i sum_d T_di d/dX_di W(r_j - X_i)  (forward mode of App. C's scatter)."""
    M = n ** 3
    rho = np.zeros(M)
    for idx, _, grad in _tap_products(X, n, L, order, shift):
        rho += np.bincount(idx, weights=T[0] * grad[0] + T[1] * grad[1] + T[2] * grad[2], minlength=M)
    return rho.reshape(n, n, n)


# --------------------------------------------------------------------------
# NUFFT force (Sec. 2.5, force evaluation with the non-uniform FFT)
# --------------------------------------------------------------------------

ES_WIDTH = 5                    # kernel support in fine-grid cells (5^3 taps)
ES_BETA = 2.30 * ES_WIDTH       # shape parameter for a grid upsampled twice


def es_kernel(t):
    """Exponential-of-semicircle kernel exp(beta (sqrt(1 - z^2) - 1)), z = 2 t / w,
    zero for |z| > 1 (t in fine-grid cells)."""
    z = 2.0 * np.asarray(t, dtype=np.float64) / ES_WIDTH
    return np.where(np.abs(z) <= 1.0, np.exp(ES_BETA * (np.sqrt(np.maximum(1.0 - z * z, 0.0)) - 1.0)), 0.0)


def es_taps(u):
    """The ES kernel's 5 cells around u (cells): nearest node i0 = floor(u + 1/2)
    and its neighbours at -2..2, with their weights."""
    i0 = np.floor(np.asarray(u) + 0.5).astype(np.int64)
    return [(i0 + o, es_kernel(i0 + o - u)) for o in range(-2, 3)]


def es_fourier(nf):
    """Continuous transform of the ES kernel at the DFT frequencies of an nf-cell
    axis, int phi(t) cos(kappa t) dt with kappa = 2 pi m / nf (adaptive quadrature)."""
    from scipy import integrate
    mf = np.fft.fftfreq(nf, 1.0 / nf)
    half = ES_WIDTH / 2.0
    return np.array([integrate.quad(lambda t: float(es_kernel(t)) * math.cos(2 * math.pi * m / nf * t),
                                    -half, half, limit=400, epsabs=1e-14, epsrel=1e-12)[0] for m in mf])


def nufft_force(X, n, L):
    """Force at the particles by the NUFFT (type 1 then type 2) on a grid upsampled
    twice, nf = 2 n: spread unit masses with the ES kernel, FFT, keep the modes with
    |m_c| < n/2 on every axis, multiply by the exact m_c = -i k_c / (-k^2) and by
    1/psi^(k)^2 (psi^ = prod of es_fourier: once for the spreading, once for the
    interpolation back), inverse FFT with scale 1/N, interpolate with the ES kernel.
    Approximates nufft_band_force to the kernel's accuracy.  X: (3, N)."""
    N = X.shape[1]
    nf = 2 * n
    H = L / nf
    t3 = [es_taps(X[c] / H) for c in range(3)]
    rho = np.zeros((nf, nf, nf))
    for iz, wz in t3[2]:
        for iy, wy in t3[1]:
            for ix, wx in t3[0]:
                np.add.at(rho, (iz % nf, iy % nf, ix % nf), wz * wy * wx)
    mf = np.fft.fftfreq(nf, 1.0 / nf)
    dec = np.where(np.abs(mf) < n / 2, 1.0 / es_fourier(nf) ** 2, 0.0)
    k1 = 2.0 * math.pi / L * mf
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(k2 > 0, 1.0 / k2, 0.0)
    D = dec[:, None, None] * dec[None, :, None] * dec[None, None, :]
    rk = np.fft.fftn(rho)
    out = np.zeros((3, N))
    for c, kc in enumerate((kx, ky, kz)):
        g = np.fft.ifftn(1j * kc * inv * D * rk).real * nf ** 3 / N
        acc = np.zeros(N)
        for iz, wz in t3[2]:
            for iy, wy in t3[1]:
                for ix, wx in t3[0]:
                    acc += wz * wy * wx * g[iz % nf, iy % nf, ix % nf]
        out[c] = acc
    return out


def density_contrast(X, n, L, order, shift=0.0):
    """delta_j = rho_j M / N - 1 with unit particle masses (Sec. 2.5, Fourier density with PM)."""
    N = X.shape[1]
    return scatter(X, None, n, L, order, shift) * (n ** 3 / N) - 1.0


# --------------------------------------------------------------------------
# Fourier-space derivative kernels, Table 2
# --------------------------------------------------------------------------

def wavenumbers(n, L):
    """Per-axis wavenumbers k = 2 pi m / L, m = 0..n/2-1, -n/2..-1 (index n/2 is
    the Nyquist mode, taken as -k_Ny)."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    return 2.0 * math.pi / L * m


def grad_kernel_1d(k, H, order):
    """Fourier transform of the 1D gradient of Table 2 (physical units).

    Table 2 gives the kernels for kt = k / k_Ny, k_Ny = pi / H; multiplying by
    k_Ny converts to physical units.
    """
    kny = math.pi / H
    kt = k / kny
    if order == 0:
        return 1j * k
    if order == 2:
        return 1j / math.pi * np.sin(math.pi * kt) * kny
    if order == 4:
        return 1j / (6.0 * math.pi) * (-np.sin(2 * math.pi * kt) + 8.0 * np.sin(math.pi * kt)) * kny
    if order == 6:
        return 1j / (30.0 * math.pi) * (np.sin(3 * math.pi * kt) - 9.0 * np.sin(2 * math.pi * kt)
                                        + 45.0 * np.sin(math.pi * kt)) * kny
    raise ValueError(order)


def laplace_kernel_1d(k, H, order):
    """Fourier transform of the 1D second derivative of Table 2 (physical units).

    Reading: the order-2 entry is printed as -(2/pi^2)[cos(pi k) - 1], which is
    positive and tends to +k^2; the stencil [1 -2 1] transforms to
    +(2/pi^2)[cos(pi k) - 1] (tending to -k^2 like the order-4 and order-6
    entries), which is what is used here.
    """
    kny = math.pi / H
    kt = k / kny
    c1, c2, c3 = np.cos(math.pi * kt), np.cos(2 * math.pi * kt), np.cos(3 * math.pi * kt)
    if order == 0:
        return -k * k
    if order == 2:
        return (2.0 / math.pi ** 2) * (c1 - 1.0) * kny ** 2
    if order == 4:
        return -(1.0 / (6.0 * math.pi ** 2)) * (c2 - 16.0 * c1 + 15.0) * kny ** 2
    if order == 6:
        return -(1.0 / (90.0 * math.pi ** 2)) * (-2.0 * c3 + 27.0 * c2 - 270.0 * c1 + 245.0) * kny ** 2
    raise ValueError(order)


def kernel_fourier_1d(k, H, order):
    """Fourier transform of the 1D mass assignment kernel of order p (Table 1):
    W^(k) = sinc^p(kt / 2) with sinc(x) = sin(pi x)/(pi x) and kt = k / k_Ny,
    k_Ny = pi / H (the table's units), i.e. [sin(k H/2) / (k H/2)]^p."""
    kt = k / (math.pi / H)
    return np.sinc(0.5 * kt) ** order


def deconvolution_1d(k, H, order):
    """1 / W^(k)^2 per axis: dividing the density by the squared kernel undoes the
    smoothing of the deposit and of the interpolation back to the particles
    (Sec. 2.5, deconvolution of the interpolation kernel).  Finite up to the
    Nyquist mode, where W^ = (2/pi)^p."""
    return 1.0 / kernel_fourier_1d(k, H, order) ** 2


def force_multipliers(n, L, grad_order, lap_order, zero_all_nyquist=False, deconvolve_order=0):
    """m_c(k) with g_c^ = m_c delta^, i.e. g = -grad Lap^-1 delta (Sec. 2.5, Computing the forces).

    phi^ = delta^ / K_lap(k),  g_c^ = -D1(k_c) phi^.
    Reading of "3D kernels are the product of the 1D kernels" for derivatives:
    K_lap(k) = sum_c L1(k_c) and the c-component of the gradient uses D1(k_c).
    The k = 0 mode is set to zero.  The gradient of component c is set to zero
    on its Nyquist plane (k_c = n/2), where an odd kernel cannot give a real
    field.  With ``zero_all_nyquist`` every mode on any Nyquist plane is zeroed
    (used with interlacing, whose half-cell phase is not Hermitian there).
    ``deconvolve_order`` p > 0 also divides by the squared 3D kernel, the product
    over the axes of W^(k_c)^2 for the order-p kernel.
    Returns a list of 3 complex arrays of shape (n, n, n) [z, y, x].
    """
    H = L / n
    k1 = wavenumbers(n, L)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = (kx, ky, kz)
    lap = sum(laplace_kernel_1d(kc, H, lap_order) for kc in kk)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv_lap = np.where(lap != 0.0, 1.0 / lap, 0.0)
    inv_lap[0, 0, 0] = 0.0
    if deconvolve_order:
        inv_lap = inv_lap * np.prod([deconvolution_1d(kc, H, deconvolve_order) for kc in kk], axis=0)
    idx = np.arange(n)
    nyq = (idx == n // 2)
    nz, ny, nx = np.meshgrid(nyq, nyq, nyq, indexing="ij")
    nyq_c = (nx, ny, nz)
    any_nyq = nx | ny | nz
    ms = []
    for c in range(3):
        m = -grad_kernel_1d(kk[c], H, grad_order) * inv_lap
        m = np.where(nyq_c[c], 0.0, m)
        if zero_all_nyquist:
            m = np.where(any_nyq, 0.0, m)
        ms.append(m)
    return ms


def apply_multiplier(field, m):
    """Real-space linear operator with Fourier multiplier m: Re IDFT(m DFT(field)).
    The imaginary part is checked to be round-off."""
    out = np.fft.ifftn(m * np.fft.fftn(field))
    assert np.max(np.abs(out.imag)) <= 1e-9 * (1.0 + np.max(np.abs(out.real))), "non-Hermitian multiplier"
    return out.real


def force_field(delta, L, grad_order, lap_order, deconvolve_order=0):
    """g_c = -d_c Lap^-1 delta on the mesh (units of length), c = x, y, z;
    deconvolve_order p > 0 first divides delta^ by the squared order-p kernel."""
    n = delta.shape[0]
    return [apply_multiplier(delta, m)
            for m in force_multipliers(n, L, grad_order, lap_order, deconvolve_order=deconvolve_order)]


def interlace_phase(n, L, sign):
    """exp(sign * i k.s) with s = (H/2)(1,1,1)."""
    H = L / n
    k1 = wavenumbers(n, L)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    return np.exp(sign * 1j * (kx + ky + kz) * 0.5 * H)


# --------------------------------------------------------------------------
# Power spectrum (Sec. 2.9, analysis)
# --------------------------------------------------------------------------

def power_spectrum(delta, L, n_bins):
    """Binned P(k) = (L^3 / M^2) <|delta^_k|^2> over every mode of the full
    n^3 DFT grid.  Reading (the paper gives no estimator details): bin b holds
    modes with (b + 1/2) k_F <= |k| < (b + 3/2) k_F, k_F = 2 pi / L; no
    deconvolution and no shot-noise subtraction; k_mean is the mean |k| of the
    bin's modes.  Returns (k_mean, P, n_modes)."""
    n = delta.shape[0]
    M = n ** 3
    dk = np.fft.fftn(delta)
    k1 = wavenumbers(n, L)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2).reshape(-1)
    kf = 2.0 * math.pi / L
    b = np.floor(kmag / kf - 0.5).astype(np.int64)
    p = (np.abs(dk) ** 2).reshape(-1)
    sel = (b >= 0) & (b < n_bins)
    cnt = np.bincount(b[sel], minlength=n_bins)
    psum = np.bincount(b[sel], weights=p[sel], minlength=n_bins)
    ksum = np.bincount(b[sel], weights=kmag[sel], minlength=n_bins)
    with np.errstate(invalid="ignore", divide="ignore"):
        kmean = np.where(cnt > 0, ksum / np.maximum(cnt, 1), 0.0)
        pk = np.where(cnt > 0, psum / np.maximum(cnt, 1) * L ** 3 / M ** 2, 0.0)
    return kmean, pk, cnt
