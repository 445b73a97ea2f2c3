"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

Holds none of the method's arithmetic: only random draws and the lattice
ordering convention (particle i = (iz n + iy) n + ix, arrays indexed [z, y, x]).
"""
import numpy as np


def white_noise(n, seed, batch=None):
    """Unit-variance Gaussian white noise on an n^3 lattice (float64), shape
    (n, n, n) or (batch, n, n, n) with seeds seed, seed+1, ..."""
    if batch is None:
        return np.random.default_rng(seed).standard_normal((n, n, n))
    return np.stack([np.random.default_rng(seed + b).standard_normal((n, n, n)) for b in range(batch)])


def random_displacements(n, scale, seed):
    """Gaussian displacements of shape (3, n^3) with standard deviation `scale`."""
    return np.random.default_rng(seed).normal(scale=scale, size=(3, n ** 3))


def random_field(n, seed, scale=1.0):
    return np.random.default_rng(seed).normal(scale=scale, size=(n, n, n))


def structured_displacements(n, cell, seed):
    """Displacements (3, n^3) that exercise the tiled particle kernels' paths:
    sub-cell jitter around the lattice (columns that keep their cells), whole
    z-columns collapsed onto one cell (several particles per cell), and a sparse
    set of particles thrown 5-20 cells away (outside any tile window), each a
    third of the lattice rows in y.  `cell` is the mesh spacing."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(-0.45, 0.45, size=(3, n, n, n)) * cell           # [c, z, y, x]
    iz = np.arange(n)[:, None, None]
    rows = np.arange(n)[None, :, None] % 3
    collapse = np.broadcast_to(rows == 1, (n, n, n))
    # collapse each run of 8 lattice planes onto the run's middle plane (+ jitter)
    d[2] = np.where(collapse, (4 - (iz % 8) - 0.5) * cell + 0.2 * d[2], d[2])
    far = (rows == 2) & (rng.random((n, n, n)) < 0.05)
    jump = rng.choice([-1.0, 1.0], size=(3, n, n, n)) * rng.uniform(5.0, 20.0, size=(3, n, n, n)) * cell
    d = np.where(far[None], d + jump, d)
    return d.reshape(3, -1)
