"""Integer-exact phase maps (uint16, indexed [x, y, z]).

Coordinates are kept in units of 1/256 voxel as int64.  The centre of voxel
j along an axis sits at (2j+1)/2 voxels = (2j+1)*128 lattice units.
"""

import numpy as np

from .draws import LATTICE, uniform_seeds

HALF = LATTICE // 2


def _centres(n):
    return (2 * np.arange(n, dtype=np.int64) + 1) * HALF


def centred_sphere(n, radius_vox, inside_phase=1, outside_phase=0):
    """Sphere of the given radius (voxels) centred in the box; membership inclusive.

    A voxel is inside iff sum_a (2 j_a + 1 - n_a)^2 <= (2 r)^2, i.e. its centre
    lies within r voxels of the box centre.
    """
    n = tuple(int(v) for v in n)
    g = [2 * np.arange(v, dtype=np.int64) + 1 - v for v in n]
    d2 = g[0][:, None, None] ** 2 + g[1][None, :, None] ** 2 + g[2][None, None, :] ** 2
    if not float(radius_vox).is_integer():
        raise ValueError("radius must be an integer number of voxels")
    inside = d2 <= (2 * int(radius_vox)) ** 2
    out = np.full(n, outside_phase, dtype=np.uint16)
    out[inside] = inside_phase
    return out


def voronoi(n, n_seeds, seed):
    """Voronoi tessellation of the box (non-periodic Euclidean distance).

    Seeds are drawn by :func:`uniform_seeds`.  Squared distances from voxel
    centres to seeds are exact int64; ties go to the lowest seed index.
    Returns (phase map uint16, seed coordinates int64).
    """
    n = tuple(int(v) for v in n)
    seeds = uniform_seeds(n_seeds, n, seed)
    cx, cy, cz = (_centres(v) for v in n)
    out = np.empty(n, dtype=np.uint16)
    # Exact search, one x-slab at a time, candidates pruned with a kd-tree
    # over float64 copies (coordinates < 2^17, squared sums < 2^53: exact).
    from scipy.spatial import cKDTree

    tree = cKDTree(seeds.astype(np.float64))
    k = min(8, n_seeds)
    yy, zz = np.meshgrid(cy, cz, indexing="ij")
    for i, x in enumerate(cx):
        pts = np.stack([np.full(yy.size, x), yy.ravel(), zz.ravel()], axis=1)
        _, idx = tree.query(pts.astype(np.float64), k=k)
        idx = np.asarray(idx).reshape(pts.shape[0], k)
        cand = seeds[idx]  # (m, k, 3) int64
        d2 = ((cand - pts[:, None, :]) ** 2).sum(axis=2)
        best = d2.min(axis=1)
        # every seed at the minimal exact distance must be among the k found
        if k < n_seeds and np.any(d2[:, -1] == best):
            raise RuntimeError("voronoi: tie wider than the candidate set")
        idx_masked = np.where(d2 == best[:, None], idx, np.iinfo(np.int64).max)
        out[i] = idx_masked.min(axis=1).reshape(yy.shape).astype(np.uint16)
    return out, seeds


def random_spheres(n, fraction, r_min, r_max, seed, inside_phase=1, outside_phase=0):
    """Overlapping random spheres added until the voxel fraction reaches `fraction`.

    Centres uniform on the 1/256 lattice, radii uniform in [r_min, r_max] voxels
    on the same lattice; membership is inclusive (exact int64 test).  Sphere
    placement stops at the first sphere that brings the inside fraction to
    >= `fraction`.
    """
    n = tuple(int(v) for v in n)
    rng = np.random.default_rng(seed)
    cx, cy, cz = (_centres(v) for v in n)
    inside = np.zeros(n, dtype=bool)
    target = fraction * inside.size
    count = 0
    while inside.sum() < target:
        c = rng.integers(0, np.asarray(n, dtype=np.int64) * LATTICE, size=3, dtype=np.int64)
        r = rng.integers(int(r_min * LATTICE), int(r_max * LATTICE) + 1, dtype=np.int64)
        lo = [max(0, int((c[a] - r) // LATTICE) - 1) for a in range(3)]
        hi = [min(n[a], int((c[a] + r) // LATTICE) + 2) for a in range(3)]
        dx = (cx[lo[0]:hi[0]] - c[0]) ** 2
        dy = (cy[lo[1]:hi[1]] - c[1]) ** 2
        dz = (cz[lo[2]:hi[2]] - c[2]) ** 2
        d2 = dx[:, None, None] + dy[None, :, None] + dz[None, None, :]
        inside[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] |= d2 <= r * r
        count += 1
        if count > 100000:
            raise RuntimeError("random_spheres: did not reach the target fraction")
    out = np.full(n, outside_phase, dtype=np.uint16)
    out[inside] = inside_phase
    return out


def laminate(n, axis, period, phases=(0, 1)):
    """Layers normal to `axis`; voxel j belongs to phases[(j // period) % len(phases)]."""
    n = tuple(int(v) for v in n)
    j = np.arange(n[axis])
    layer = np.asarray(phases, dtype=np.uint16)[(j // period) % len(phases)]
    shape = [1, 1, 1]
    shape[axis] = n[axis]
    return np.broadcast_to(layer.reshape(shape), n).copy()
