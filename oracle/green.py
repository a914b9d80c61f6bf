"""B0, 2mu0 and C0 discrete Green operators (Sec. 2.6.1, Sec. 2.6.2, Sec. 2.6.3).

Per component i (no summation), Eq. NSGO2_HEX1 / NSGO2_TETRA2:

    u^f_i = - p_i / (2 mu0 ||xi||^2 + lambda0 |xi_i|^2)

with the modified frequency vector of the scheme built from the fundamental
frequencies of component i's own transforms (Table 1, Sec. 2.5.1 "Derivation
in Fourier space"):

    HEX1  (xi_H)_a = (2/h_a) sin(xi_a/2) prod_{b != a} cos(xi_b/2)        (Eq. modified_freq_hex1)
    TETRA2 xi_T1 = xi_H - i xi', (xi')_a = (2/h_a) cos(xi_a/2) prod_{b != a} sin(xi_b/2)
           (Eq. freq_TETRA2), xi_T2 = conj(xi_T1), so |xi_T2,a|^2 = (xi_H)_a^2 + (xi')_a^2.

The 2mu0 operator (Eqs. NSGO1_HEX1, NSGO1_TETRA2) is the case lambda0 = 0.
A null denominator gives u^f = 0 (Sec. 2.6, after Eq. NSGO2_TETRA2); nullness
is decided with exact half-angle zeros (see bc.half_angles).
"""

import numpy as np

from .bc import half_angles


def squared_symbols(kinds, n, h, scheme):
    """Per-axis squared modified-frequency components |xi_a|^2 on the 3D frequency grid."""
    s = []
    c = []
    for a in range(3):
        sa, ca = half_angles(kinds[a], n[a])
        shape = [1, 1, 1]
        shape[a] = sa.size
        s.append(sa.reshape(shape))
        c.append(ca.reshape(shape))
    sq = []
    for a in range(3):
        b, d = [x for x in range(3) if x != a]
        xh = (2.0 / h[a]) * s[a] * c[b] * c[d]
        val = xh * xh
        if scheme == "TETRA2":
            xp = (2.0 / h[a]) * c[a] * s[b] * s[d]
            val = val + xp * xp
        sq.append(val)
    return [np.broadcast_to(v, np.broadcast_shapes(*[x.shape for x in sq])) for v in sq]


def green_factor(grid, q, scheme, lambda0, mu0):
    """Real factor g such that u^f_q = g * p_q on component q's frequency grid (0 where null)."""
    sq = squared_symbols(grid.kind[q], grid.n, grid.h, scheme)
    den = 2.0 * mu0 * (sq[0] + sq[1] + sq[2]) + lambda0 * sq[q]
    g = np.zeros(den.shape)
    nz = den != 0.0
    g[nz] = -1.0 / den[nz]
    return g


def operator_symbol(grid, q, scheme, lambda0, mu0):
    """Symbol of div(B0 : grad u)_q on component q's frequency grid: -(2mu0 ||xi||^2 + lambda0 |xi_q|^2)."""
    sq = squared_symbols(grid.kind[q], grid.n, grid.h, scheme)
    return -(2.0 * mu0 * (sq[0] + sq[1] + sq[2]) + lambda0 * sq[q])


# ---- the C0 discrete Green operator (Sec. 2.6.1), HEX1, normal-mixed BCs -------------------
# R0 : grad u = C0 : grad u = 2 mu0 grad u + lambda0 tr(grad u) 1 (Eq. TF_C0_behavior), so
# div(R0 : grad u) = 2 mu0 div grad u + lambda0 div grad^T u (Eq. FourierSGO), which couples the
# three components.  With HEX1 the symbol is -(2 mu0 |xi_H|^2 I + lambda0 xi_H (x) xi_H) and its
# inverse is Eq. FourierSGO_HEX1 (a rank-one correction of the diagonal part).
#
# Reading (the paper states it in the Fourier space of the extended fields): on the real
# DCT-I / DST-I coefficients the library and this oracle use, a derivative along axis a maps
# the cosine series of a symmetric component to the sine series of the opposite parity and
# back, with the factor -(2/h_a) sin(xi_a/2) (cosine -> sine) or +(2/h_a) sin(xi_a/2) (sine ->
# cosine), and the averages of the HEX1 stencil give the cos(xi_b/2) factors; for normal-mixed
# BCs (Eq. SGO_BCs) the coupling term lambda0 D_q D_i u_i lands on u_q's own series at the same
# node position, so the symbol on the real coefficients is -(2 mu0 |xi_H|^2 I + lambda0 v (x) v)
# with v_q = tau_q (xi_H)_q, tau_q = -1 when u_q is symmetric about the faces normal to q
# (DCT-I along q) and +1 when it is anti-symmetric (DST-I).  The real-space operator pins this
# (tests/test_oracle_c0.py).
#
# TETRA2 (Eqs. p_u_tetra2, FourierSGO_TETRA2_1/2): with xi_T2 = xi_H + i xi' (Eq. freq_TETRA2) the
# symbol is -(2 mu0 |xi_T2|^2 I + lambda0/2 [xi_T2 (x) conj(xi_T2) + conj(xi_T2) (x) xi_T2]), on the
# real coefficients -(2 mu0 |z|^2 I + lambda0/2 [z (x) conj(z) + conj(z) (x) z]) with z = v + i w,
# w_q = tau_q xi'_q (the same signs; the real-space operator pins it).  Its inverse follows the
# paper's steps: the dot products of p with z and conj(z), the 2 x 2 system for u . z and
# u . conj(z) obtained by dotting the operator with z and conj(z), then back-substitution.  Reading
# taken: the diagonal coefficient of that system is taken from the operator itself,
# 2 mu0 + lambda0 / 2 = (4 mu0 + lambda0) / 2 times |z|^2 -- the printed (2 mu0 + lambda0) / 2 would
# not reduce to Eq. FourierSGO_HEX1 when xi' = 0, while this one does.
#
# Supported here: every axis non-periodic with the same symmetries on both faces (no
# quarter-wave kinds); on each axis the normal component's symmetry opposite to the tangential
# ones'.

def c0_unsupported(grid, scheme):
    """None if the C0 operator below applies to this grid, else the reason."""
    if scheme not in ("HEX1", "TETRA2"):
        return "unknown scheme"
    for a in range(3):
        for q in range(3):
            k = grid.kind[q][a]
            if k not in ("DCT1", "DST1"):
                return "C0 needs non-periodic axes with the same symmetry on both faces"
        normal = grid.kind[a][a]
        for q in range(3):
            if q != a and grid.kind[q][a] == normal:
                return "C0 needs normal-mixed BCs (Eq. SGO_BCs): normal and tangential symmetries opposite"
    return None


def c0_vectors(grid, scheme="HEX1"):
    """(v[3], w[3], |xi|^2) on the node positions m (xi_a = pi m_a / n_a for DCT-I and DST-I
    alike); w = 0 for HEX1, |xi|^2 = |xi_H|^2 + |xi'|^2 for TETRA2."""
    s, c = [], []
    for a in range(3):
        sa, ca = half_angles("DCT1", grid.n[a])  # positions 0..n, exact zeros at both ends
        shape = [1, 1, 1]
        shape[a] = sa.size
        s.append(sa.reshape(shape))
        c.append(ca.reshape(shape))
    xi, xp = [], []
    for a in range(3):
        b, d = [x for x in range(3) if x != a]
        xi.append((2.0 / grid.h[a]) * s[a] * c[b] * c[d])
        xp.append((2.0 / grid.h[a]) * c[a] * s[b] * s[d] if scheme == "TETRA2" else 0.0 * s[a])
    shape = np.broadcast_shapes(*[x.shape for x in xi + xp])
    xi = [np.broadcast_to(x, shape) for x in xi]
    xp = [np.broadcast_to(x, shape) for x in xp]
    xx = sum(xi[q] ** 2 + xp[q] ** 2 for q in range(3))
    tau = [-1.0 if grid.kind[q][q] == "DCT1" else 1.0 for q in range(3)]
    return [tau[q] * xi[q] for q in range(3)], [tau[q] * xp[q] for q in range(3)], xx


def c0_symbol_apply(grid, lambda0, mu0, uhat, scheme="HEX1"):
    """p_hat = -(2 mu0 |xi|^2 u_hat + lambda0 [(v . u_hat) v + (w . u_hat) w]) on node positions."""
    v, w, xx = c0_vectors(grid, scheme)
    vu = sum(v[q] * uhat[q] for q in range(3))
    wu = sum(w[q] * uhat[q] for q in range(3))
    return [-(2.0 * mu0 * xx * uhat[q] + lambda0 * (vu * v[q] + wu * w[q])) for q in range(3)]


def c0_green_apply(grid, lambda0, mu0, phat, scheme="HEX1"):
    """The C0 discrete Green operator on the real coefficients, zero where |xi|^2 = 0 (the null
    rule of Sec. 2.6).  HEX1, Eq. FourierSGO_HEX1: u_hat = -(p_hat - lambda0 / (2 mu0 + lambda0)
    (v . p_hat) v / |xi|^2) / (2 mu0 |xi|^2).  TETRA2, Eqs. FourierSGO_TETRA2_1/2 with z = v + i w
    and the reading of its diagonal coefficient stated above."""
    v, w, xx = c0_vectors(grid, scheme)
    nz = xx > 0.0
    safe = np.where(nz, xx, 1.0)
    if scheme == "HEX1":
        vp = sum(v[q] * phat[q] for q in range(3))
        beta = lambda0 / (2.0 * mu0 + lambda0)
        return [np.where(nz, -(phat[q] - beta * vp * v[q] / safe) / (2.0 * mu0 * safe), 0.0) for q in range(3)]
    z = [v[q] + 1j * w[q] for q in range(3)]
    zc = [np.conj(zq) for zq in z]
    pz = sum(phat[q] * z[q] for q in range(3))      # p . z
    pzc = sum(phat[q] * zc[q] for q in range(3))    # p . conj(z)
    zz = sum(zq * zq for zq in z)                   # z . z
    zzc = np.conj(zz)                               # conj(z) . conj(z)
    d = (2.0 * mu0 + 0.5 * lambda0) * safe          # the diagonal coefficient (read above) times |z|^2
    Ds = d * d - (0.5 * lambda0) ** 2 * np.abs(zz) ** 2
    Ds = np.where(nz, Ds, 1.0)
    # u . z and u . conj(z) from  -p.z = d (u.z) + lambda0/2 (z.z) (u.conj z)  and its conjugate pair
    p_int1 = (-d * pz + 0.5 * lambda0 * zz * pzc) / Ds   # = u . z
    p_int2 = (0.5 * lambda0 * zzc * pz - d * pzc) / Ds   # = u . conj(z)
    out = []
    for q in range(3):
        uq = -(phat[q] + 0.5 * lambda0 * (p_int2 * z[q] + p_int1 * zc[q])) / (2.0 * mu0 * safe)
        out.append(np.where(nz, np.real(uq), 0.0))
    return out
