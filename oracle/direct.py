"""The discrete linear-elastic problem solved directly (a pin for the fixed point).

For a linear law the problem of Eq. GeneralBCtobesolved is a sparse linear
system.  It is assembled here as a finite-element-like stiffness, independent
of the ghost-voxel code in ``stencils``: the gradient is a sparse matrix B
from the transformed node components (Dirichlet nodes removed, periodic nodes
identified) to the voxel-point gradients (Eqs. D1HG-D3HG / D1T1T2G-D3T1T2G),
and the residual of the method satisfies D = W^-1 (-B^T P / n_ppv) with W the
nodal weights (1/2 per non-periodic face a node lies on).  So D = 0 is

    K u = f,   K = B^T Cblk B / n_ppv,   f = -B^T Cblk G* / n_ppv,

solved with SciPy's SuperLU.  Only for grids without null modes of K.
"""

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .bc import Grid, dof_range
from .laws import B0_LINEAR, CUBIC_ELASTIC, ISO_ELASTIC, iso_tensor, rotated_cubic

_HEX = [[(o, 1.0 if o[i] else -1.0) for o in itertools.product((0, 1), repeat=3)] for i in range(3)]
_TET = [
    [  # T1, rows i = 0, 1, 2 (Eqs. D1T1T2G-D3T1T2G, first lines)
        [((1, 1, 0), 1.0), ((0, 1, 1), -1.0), ((1, 0, 1), 1.0), ((0, 0, 0), -1.0)],
        [((1, 1, 0), 1.0), ((0, 0, 0), -1.0), ((0, 1, 1), 1.0), ((1, 0, 1), -1.0)],
        [((0, 1, 1), 1.0), ((0, 0, 0), -1.0), ((1, 0, 1), 1.0), ((1, 1, 0), -1.0)],
    ],
    [  # T2 (second lines)
        [((1, 0, 0), 1.0), ((0, 0, 1), -1.0), ((1, 1, 1), 1.0), ((0, 1, 0), -1.0)],
        [((0, 1, 0), 1.0), ((1, 0, 0), -1.0), ((1, 1, 1), 1.0), ((0, 0, 1), -1.0)],
        [((0, 0, 1), 1.0), ((0, 1, 0), -1.0), ((1, 1, 1), 1.0), ((1, 0, 0), -1.0)],
    ],
]


def dof_numbering(grid):
    """index[q] (N1,N2,N3) int array: DOF number, or -1 for a dismissed node."""
    idx = []
    count = 0
    for q in range(3):
        a = -np.ones(grid.N, dtype=np.int64)
        sl = tuple(slice(*dof_range(grid.kind[q][ax], grid.n[ax])) for ax in range(3))
        m = np.zeros(grid.N, dtype=bool)
        m[sl] = True
        k = int(m.sum())
        a[m] = np.arange(count, count + k)
        count += k
        idx.append(a)
    return idx, count


def gradient_matrix(grid, scheme):
    """Sparse B: DOF vector -> G[r, i, q, voxel] (row-major over (r, i, q, x, y, z))."""
    idx, ndof = dof_numbering(grid)
    n = grid.n
    nv = n[0] * n[1] * n[2]
    tabs, scale = ([_HEX], 0.25) if scheme == "HEX1" else (_TET, 0.5)
    vx, vy, vz = np.meshgrid(*[np.arange(v) for v in n], indexing="ij")
    vflat = np.arange(nv)
    rows, cols, vals = [], [], []
    for r, tab in enumerate(tabs):
        for i in range(3):
            for o, s in tab[i]:
                nx, ny, nz = vx + o[0], vy + o[1], vz + o[2]
                if grid.periodic[0]:
                    nx = nx % n[0]
                if grid.periodic[1]:
                    ny = ny % n[1]
                if grid.periodic[2]:
                    nz = nz % n[2]
                for q in range(3):
                    c = idx[q][nx, ny, nz].ravel()
                    keep = c >= 0
                    row = ((r * 3 + i) * 3 + q) * nv + vflat
                    rows.append(row[keep])
                    cols.append(c[keep])
                    vals.append(np.full(int(keep.sum()), s * scale / grid.h[i]))
    B = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(len(tabs) * 9 * nv, ndof))
    return B, idx, ndof


def _stiffness_9x9(mat):
    if mat.law == ISO_ELASTIC:
        C = iso_tensor(*mat.params[:2])
    elif mat.law == CUBIC_ELASTIC:
        C = rotated_cubic(mat.params[:3], mat.quat)
    elif mat.law == B0_LINEAR:
        lam, mu = mat.params[:2]
        C = np.zeros((3, 3, 3, 3))
        for i in range(3):
            for q in range(3):
                C[i, q, i, q] += 2 * mu
            C[i, i, i, i] += lam
    else:
        raise ValueError("direct solve needs a linear law")
    # P_iq = C_iqkl G_kl for every law here (minor symmetry, or the B0 law itself)
    return C.reshape(9, 9)


def material_block(wl, npp):
    """Block-diagonal map G -> P over (r, i, q, voxel) rows."""
    n = wl.phase.shape
    nv = int(np.prod(n))
    ph = np.asarray(wl.phase).ravel()
    Cs = np.stack([_stiffness_9x9(m) for m in wl.materials])  # (nph, 9, 9)
    rows, cols, vals = [], [], []
    vflat = np.arange(nv)
    for r in range(npp):
        for a in range(9):
            for b in range(9):
                v = Cs[ph, a, b]
                keep = v != 0.0
                rows.append((r * 9 + a) * nv + vflat[keep])
                cols.append((r * 9 + b) * nv + vflat[keep])
                vals.append(v[keep])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(npp * 9 * nv, npp * 9 * nv))


def solve(wl, Gstar):
    """Solve K u = f; returns u^f on the stored node grid (3, N1, N2, N3)."""
    grid = Grid(wl.n, wl.bc, wl.h)
    npp = 1 if wl.scheme == "HEX1" else 2
    B, idx, ndof = gradient_matrix(grid, wl.scheme)
    C = material_block(wl, npp)
    K = (B.T @ C @ B) / npp
    f = -(B.T @ (C @ np.asarray(Gstar).reshape(-1))) / npp
    x = spla.spsolve(K.tocsc(), f)
    u = np.zeros((3,) + grid.N)
    for q in range(3):
        m = idx[q] >= 0
        u[q][m] = x[idx[q][m]]
    return u
