"""Seeded random draws (inputs only)."""

import numpy as np

LATTICE = 256  # sub-voxel lattice used for seed / centre coordinates


def uniform_seeds(n_seeds, n, seed):
    """Integer seed points uniform in the box [0, n_a) voxels, on a 1/256 lattice.

    Returns an int64 array (n_seeds, 3) of coordinates in units of 1/256 voxel.
    """
    rng = np.random.default_rng(seed)
    n = np.asarray(n, dtype=np.int64)
    return rng.integers(0, n * LATTICE, size=(n_seeds, 3), dtype=np.int64)


def shoemake_quaternions(count, seed):
    """Unit quaternions uniform on SO(3) (Shoemake, Graphics Gems III, 1992).

    Returned as (w, x, y, z) rows, float64.
    """
    rng = np.random.default_rng(seed)
    u = rng.random((count, 3))
    a = np.sqrt(1.0 - u[:, 0])
    b = np.sqrt(u[:, 0])
    t1 = 2.0 * np.pi * u[:, 1]
    t2 = 2.0 * np.pi * u[:, 2]
    q = np.stack([b * np.cos(t2), a * np.sin(t1), a * np.cos(t1), b * np.sin(t2)], axis=1)
    return q


def random_field(shape, seed, dtype=np.float64):
    """Standard-normal field of the given shape."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape).astype(dtype)
