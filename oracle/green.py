"""B0 and 2mu0 discrete Green operators (Sec. 2.6.2, Sec. 2.6.3).

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
