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
