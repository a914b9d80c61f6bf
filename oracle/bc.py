"""Boundary conditions, symmetries, node grids and frequencies.

Sec. 2.2 (Eq. GeneralBCtobesolved): a periodic face makes u^f_q periodic, a
Dirichlet condition on component q makes u^f_q anti-symmetric (A) about the
face, a Neumann condition makes it symmetric (S).  Table 1 maps each pair of
face symmetries (left, right) of a node field to one transform:

    P/P -> DFT,  S/S -> DCT-I,  S/A -> DCT-III,  A/A -> DST-I,  A/S -> DST-III

with its node index range (the other nodes are "dismissed", Sec. 2.7.2) and
its fundamental frequencies xi^k.

Node grid (Sec. 2.1, Sec. 2.7.1): a non-periodic axis with n voxels holds
n+1 nodes j = 0..n; a periodic axis stores n nodes (node n is node 0).
"""

import numpy as np

SYM_OF_BC = {"P": "P", "D": "A", "N": "S"}

KIND_OF_PAIR = {
    ("P", "P"): "DFT",
    ("S", "S"): "DCT1",
    ("S", "A"): "DCT3",
    ("A", "A"): "DST1",
    ("A", "S"): "DST3",
}

KINDS = ("DFT", "DCT1", "DCT3", "DST1", "DST3")


def dof_range(kind, n):
    """Node indices [lo, hi) a transform of this kind acts on (Table 1, index j)."""
    return {
        "DFT": (0, n),
        "DCT1": (0, n + 1),
        "DCT3": (0, n),
        "DST1": (1, n),
        "DST3": (1, n + 1),
    }[kind]


def n_freq(kind, n):
    lo, hi = dof_range(kind, n)
    return hi - lo


def frequencies(kind, n):
    """Fundamental frequencies xi^k of Table 1, with exact flags for xi = 0 and xi = pi.

    Returns (xi, is_zero, is_pi); the flags are decided on integer indices.
    """
    if kind == "DFT":
        k = np.arange(n)
        xi = 2.0 * np.pi * k / n
        return xi, k == 0, 2 * k == n
    if kind == "DCT1":
        k = np.arange(n + 1)
        xi = np.pi * k / n
        return xi, k == 0, k == n
    if kind == "DCT3" or kind == "DST3":
        k = np.arange(n)
        xi = np.pi * (k + 0.5) / n
        z = np.zeros(n, dtype=bool)
        return xi, z, z.copy()
    if kind == "DST1":
        k = np.arange(n - 1)
        xi = np.pi * (k + 1) / n
        z = np.zeros(n - 1, dtype=bool)
        return xi, z, z.copy()
    raise ValueError(kind)


def half_angles(kind, n):
    """sin(xi/2), cos(xi/2), with sin = 0 at xi = 0 and cos = 0 at xi = pi set exactly.

    The paper sets the Green operator to zero where its denominator is null
    (Sec. 2.6, after Eq. NSGO2_TETRA2); deciding nullness needs exact zeros,
    which floating-point cos(pi/2) does not give.
    """
    xi, z, p = frequencies(kind, n)
    s = np.sin(0.5 * xi)
    c = np.cos(0.5 * xi)
    s[z] = 0.0
    c[p] = 0.0
    return s, c


class Grid:
    """Voxel grid, node grid and per-component symmetries / transform kinds.

    bc[a][f][q] in {'P','D','N'}: axis a, face f (0 = contains the origin), component q.
    """

    def __init__(self, n, bc, h=(1.0, 1.0, 1.0)):
        self.n = tuple(int(v) for v in n)
        self.h = tuple(float(v) for v in h)
        self.bc = bc
        self.periodic = []
        for a in range(3):
            types = {bc[a][f][q] for f in range(2) for q in range(3)}
            if "P" in types and types != {"P"}:
                raise ValueError("a periodic axis must be periodic on both faces for all components")
            self.periodic.append(types == {"P"})
        self.N = tuple(self.n[a] if self.periodic[a] else self.n[a] + 1 for a in range(3))
        # sym[q][a] = (left, right)
        self.sym = [[(SYM_OF_BC[bc[a][0][q]], SYM_OF_BC[bc[a][1][q]]) for a in range(3)] for q in range(3)]
        self.kind = [[KIND_OF_PAIR[self.sym[q][a]] for a in range(3)] for q in range(3)]

    def dof_slices(self, q):
        return tuple(slice(*dof_range(self.kind[q][a], self.n[a])) for a in range(3))

    def dof_mask(self, q):
        m = np.zeros(self.N, dtype=bool)
        m[self.dof_slices(q)] = True
        return m

    def spectral_shape(self, q):
        return tuple(n_freq(self.kind[q][a], self.n[a]) for a in range(3))

    @property
    def node_shape(self):
        return (3,) + self.N

    @property
    def n_voxels(self):
        return self.n[0] * self.n[1] * self.n[2]
