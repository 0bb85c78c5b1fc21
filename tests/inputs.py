"""Seeded synthetic inputs shared by the oracle tests and the CUDA parity tests.

Holds none of the method's arithmetic: it only draws seeded random numbers around a
per-direction mean that the caller passes in.
"""
import numpy as np


def perturbed_populations(mean, grid_shape, seed, rel=0.1, absolute=0.0):
    """populations[a, z, y, x] = mean[a] * (1 + rel * N(0,1)) + absolute * N(0,1)"""
    rng = np.random.default_rng(seed)
    mean = np.asarray(mean, dtype=np.float64)
    shape = (mean.shape[0],) + tuple(grid_shape)
    bcast = mean.reshape((-1,) + (1,) * len(grid_shape))
    return bcast * (1.0 + rel * rng.standard_normal(shape)) + absolute * rng.standard_normal(shape)


def uniform_field(grid_shape, seed, lo, hi):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=tuple(grid_shape))


def random_rates(n, seed, lo=0.3, hi=1.9):
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def random_vectors(n, seed, scale):
    return scale * np.random.default_rng(seed).standard_normal((n, 3))
