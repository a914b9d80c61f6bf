"""Finite-difference gradient and divergence, HEX1 and TETRA2 (Sec. 2.5).

Index convention (the paper writes grad v = D_i v_j e_i (x) e_j, Sec. 2.5.1):
G[r, i, q] = D_i^{(r)} u_q at voxel point r (r = 0 for HEX1; r = 0 -> T1,
r = 1 -> T2 for TETRA2), and the divergence of a voxel tensor S is
(div S)_q = sum_i D_i S_iq at the nodes.

Node -> voxel stencils are the paper's equations written as tables of
(node offset, sign):
  HEX1   D_i = 1/(4 h_i) sum over the 8 corners o of (+1 if o_i = 1 else -1) G[j+o]
         (Eqs. D1HG-D3HG);
  TETRA2 D_i^{T1}, D_i^{T2} = 1/(2 h_i) * four signed corners (Eqs. D1T1T2G-D3T1T2G).
Voxel -> node stencils follow Remark 1: the same tables with node offsets o
replaced by centre offsets o - 1/2, so node m reads voxels m + o - 1.

TETRA2 residual: D = 1/2 (div_{T2} P^{(T1)} + div_{T1} P^{(T2)}), the pairing of
the Laplacian 1/2 (D^{T1} D^{T2} + D^{T2} D^{T1}) (Sec. 2.5.2).

Ghost voxels outside the cell (Sec. 2.7.3 "halo voxels"; Sec. 2.2): a voxel
tensor S has the symmetries of grad u^f (Eq. GeneralBCtobesolved and the
sentence after it).  Across a face normal to axis a, the ghost of S_iq is
sigma(u_q, face) * (-1 if i == a else +1) times the mirror voxel's value,
with sigma = +1 for a symmetric and -1 for an anti-symmetric u_q
(Eq. Continuous_der_symmetry_per).  For TETRA2 the mirror of tetrahedron T1
is T2 and vice versa (Sec. 2.5.2), so a ghost T1 value is taken from the
mirror's T2 value.  Periodic axes wrap.
"""

import itertools

import numpy as np

CORNERS = list(itertools.product((0, 1), repeat=3))

# HEX1 (Eqs. D1HG-D3HG): every corner, sign by the corner's coordinate along i.
HEX1 = [[(o, 1.0 if o[i] == 1 else -1.0) for o in CORNERS] for i in range(3)]
HEX1_SCALE = 0.25

# TETRA2 (Eqs. D1T1T2G, D2T1T2G, D3T1T2G), transcribed term by term.
T1 = [
    [((1, 1, 0), +1.0), ((0, 1, 1), -1.0), ((1, 0, 1), +1.0), ((0, 0, 0), -1.0)],
    [((1, 1, 0), +1.0), ((0, 0, 0), -1.0), ((0, 1, 1), +1.0), ((1, 0, 1), -1.0)],
    [((0, 1, 1), +1.0), ((0, 0, 0), -1.0), ((1, 0, 1), +1.0), ((1, 1, 0), -1.0)],
]
T2 = [
    [((1, 0, 0), +1.0), ((0, 0, 1), -1.0), ((1, 1, 1), +1.0), ((0, 1, 0), -1.0)],
    [((0, 1, 0), +1.0), ((1, 0, 0), -1.0), ((1, 1, 1), +1.0), ((0, 0, 1), -1.0)],
    [((0, 0, 1), +1.0), ((0, 1, 0), -1.0), ((1, 1, 1), +1.0), ((1, 0, 0), -1.0)],
]
T_SCALE = 0.5


def n_points(scheme):
    return 1 if scheme == "HEX1" else 2


def _tables(scheme):
    if scheme == "HEX1":
        return [HEX1], HEX1_SCALE
    if scheme == "TETRA2":
        return [T1, T2], T_SCALE
    raise ValueError(scheme)


def full_nodes(u, grid):
    """Node values on (n+1)^3 nodes: periodic axes get node n = node 0 appended."""
    x = u
    for a in range(3):
        if grid.periodic[a]:
            x = np.concatenate([x, np.take(x, [0], axis=x.ndim - 3 + a)], axis=x.ndim - 3 + a)
    return x


def grad_full(uf, grid, scheme):
    """Gradient at voxel points from node values on the full (n+1)^3 grid.

    uf: (3, n1+1, n2+1, n3+1).  Returns G (npp, 3, 3, n1, n2, n3), G[r,i,q] = D_i^{(r)} u_q.
    """
    n = grid.n
    tabs, scale = _tables(scheme)
    G = np.zeros((len(tabs), 3, 3) + n)
    for r, tab in enumerate(tabs):
        for i in range(3):
            c = scale / grid.h[i]
            for o, s in tab[i]:
                blk = uf[:, o[0]:o[0] + n[0], o[1]:o[1] + n[1], o[2]:o[2] + n[2]]
                G[r, i] += (s * c) * blk
    return G


def grad(u, grid, scheme):
    """Gradient of a node field u (3, N1, N2, N3) at the voxel points."""
    return grad_full(full_nodes(u, grid), grid, scheme)


def ghost_extend(S, grid, scheme):
    """Voxel tensor S (npp, 3, 3, n1, n2, n3) with one ghost layer on every face.

    Ghost values follow the symmetry rule in the module docstring; axes are
    processed x, y, z so edge and corner ghosts compose both reflections.
    """
    npp = S.shape[0]
    n = grid.n
    E = np.zeros(S.shape[:3] + tuple(v + 2 for v in n))
    E[..., 1:-1, 1:-1, 1:-1] = S
    swap = [1, 0] if npp == 2 else [0]
    for a in range(3):
        ax = 3 + a
        lo = [slice(None)] * 6
        hi = [slice(None)] * 6
        lo[ax] = slice(0, 1)
        hi[ax] = slice(n[a] + 1, n[a] + 2)
        first = [slice(None)] * 6
        last = [slice(None)] * 6
        first[ax] = slice(1, 2)
        last[ax] = slice(n[a], n[a] + 1)
        if grid.periodic[a]:
            E[tuple(lo)] = E[tuple(last)]
            E[tuple(hi)] = E[tuple(first)]
            continue
        for side, (dst, src) in enumerate(((lo, first), (hi, last))):
            mirror = E[tuple(src)][swap]
            sign = np.ones((3, 3))
            for q in range(3):
                sq = 1.0 if grid.sym[q][a][side] == "S" else -1.0
                for i in range(3):
                    sign[i, q] = sq * (-1.0 if i == a else 1.0)
            E[tuple(dst)] = sign[None, :, :, None, None, None] * mirror
    return E


def _div_one(Ei, tab, grid, scale):
    """sum_i D_i^{centre->node} S_iq on the stored node grid, from an extended (3,3,...) tensor."""
    N = grid.N
    out = np.zeros((3,) + N)
    for i in range(3):
        c = scale / grid.h[i]
        for o, s in tab[i]:
            # node m reads voxel m + o - 1 = extended index m + o
            blk = Ei[i, :, o[0]:o[0] + N[0], o[1]:o[1] + N[1], o[2]:o[2] + N[2]]
            out += (s * c) * blk
    return out


def _face_axes(a):
    return [b for b in range(3) if b != a]


def face_field_ghost(t, grid, a):
    """A traction field over the voxel centres of a face normal to a, t (3, n_b, n_c) with b < c
    the in-plane axes, spread over the face's whole ghost layer (extended in-plane indices
    0 .. n + 1): a ghost outside the face takes the value at the voxel it mirrors (the nearest
    face voxel on a non-periodic axis, the wrapped one on a periodic axis)."""
    b, c = _face_axes(a)
    idx = []
    for ax in (b, c):
        e = np.arange(grid.n[ax] + 2) - 1
        if grid.periodic[ax]:
            e = e % grid.n[ax]
        else:
            e = np.clip(e, 0, grid.n[ax] - 1)
        idx.append(e)
    return np.asarray(t)[:, idx[0][:, None], idx[1][None, :]]


def add_traction_ghosts(E, grid, T, Tf=None):
    """The imposed stress of non-zero Neumann tractions (Sec. 2.2, the construction of the
    Neumann-BC figure): P = P^f + P*, with P* zero inside the cell and P*_aq = 2 t_q at the
    mirror voxel centres across a face normal to axis a whose u_q is Neumann, t_q =
    (-1)^(alpha+1) T[a][alpha][q] the face value of P_aq for the traction T (outward normal
    convention, traction_q = P_iq n_i), so that P* interpolated at the face is t.  Reading:
    P* covers the whole ghost layer of the face, its edges and corners included, and is
    added after the symmetry reflections.  T: uniform tractions (or None); Tf: non-uniform
    ones, a dict {(axis, face): t (3, n_b, n_c)} over the face's voxel centres (b < c the
    in-plane axes), spread over the ghost layer by face_field_ghost and added to T."""
    n = grid.n
    for a in range(3):
        if grid.periodic[a]:
            continue
        for side in range(2):
            field = None
            if Tf is not None and (a, side) in Tf:
                field = face_field_ghost(Tf[(a, side)], grid, a)
            for q in range(3):
                t = 0.0 if T is None else T[a][side][q]
                if grid.sym[q][a][side] != "S" or (t == 0.0 and field is None):
                    continue
                idx = [slice(None)] * 6
                idx[1] = a
                idx[2] = q
                idx[3 + a] = 0 if side == 0 else n[a] + 1
                val = t if field is None else t + field[q]
                # the ghost layer slice has the two in-plane axes in order (b, c)
                E[tuple(idx)] += 2.0 * (1.0 if side == 1 else -1.0) * (val if np.ndim(val) == 0
                                                                        else val[None])
    return E


def div(S, grid, scheme, T=None, Tf=None):
    """Divergence at the nodes of a voxel tensor S (npp, 3, 3, n1, n2, n3); T: uniform
    Neumann tractions T[axis][face][component] (add_traction_ghosts) or None; Tf: per-face
    traction fields {(axis, face): t (3, n_b, n_c)} or None.

    HEX1: D_q = sum_i D_i^H S_iq.  TETRA2: 1/2 (div_{T2} S^{(T1)} + div_{T1} S^{(T2)}).
    """
    E = ghost_extend(S, grid, scheme)
    if T is not None or Tf:
        E = add_traction_ghosts(E, grid, T, Tf)
    if scheme == "HEX1":
        return _div_one(E[0], HEX1, grid, HEX1_SCALE)
    return 0.5 * (_div_one(E[0], T2, grid, T_SCALE) + _div_one(E[1], T1, grid, T_SCALE))


def node_weights(grid):
    """Quadrature weight of each stored node: 1/2 per non-periodic face the node lies on."""
    w = np.ones(grid.N)
    for a in range(3):
        if grid.periodic[a]:
            continue
        wa = np.ones(grid.N[a])
        wa[0] = wa[-1] = 0.5
        shape = [1, 1, 1]
        shape[a] = grid.N[a]
        w = w * wa.reshape(shape)
    return w
