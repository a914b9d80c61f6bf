"""The discrete transforms of Table 1 and their inverses (Sec. 2.4, Sec. 2.7.2).

Forward transforms are the Table 1 sums written out as dense matrices over the
transform's node range j (the other nodes are dismissed):

    DFT    G[k] = sum_{j=0}^{n-1} g[j] exp(-i xi_k j),                 xi_k = 2 pi k / n
    DCT-I  G[k] = sum_{j=0}^{n} (2 - d_{j0} - d_{jn}) g[j] cos(xi_k j),  xi_k = pi k / n
    DCT-III G[k] = sum_{j=0}^{n-1} (2 - d_{j0}) g[j] cos(xi_k j),        xi_k = pi (k + 1/2) / n
    DST-I  G[k] = 2 sum_{j=1}^{n-1} g[j] sin(xi_k j),                   xi_k = pi (k + 1) / n
    DST-III G[k] = sum_{j=1}^{n} (2 - d_{jn}) g[j] sin(xi_k j),          xi_k = pi (k + 1/2) / n

(n = number of voxels, N^n - 1 in the paper's notation).  The inverse of each
is, by definition, the inverse of that matrix.  A 3D DT is three 1D DTs, one
per axis (Sec. 2.7.2).  For large n the same maps are evaluated with
``scipy.fft`` (whose unnormalised DCT/DST types 1-3 are exactly these sums);
tests check the two paths against each other.

The halfcomplex real DFT used to store periodic-axis spectra as reals is
also defined here (``r2hc_matrix``): row k <= n/2 holds sum_j g[j] cos(2 pi jk/n),
row n-k (0 < k < n/2) holds -sum_j g[j] sin(2 pi jk/n).
"""

import numpy as np
import scipy.fft as sfft

from .bc import dof_range, frequencies

DENSE_MAX = 64  # dense matrices up to this n, scipy.fft above


def forward_matrix(kind, n):
    """Dense matrix of the forward transform of Table 1 (rows k, columns over the node range)."""
    xi, _, _ = frequencies(kind, n)
    lo, hi = dof_range(kind, n)
    j = np.arange(lo, hi)
    arg = np.outer(xi, j)
    if kind == "DFT":
        return np.exp(-1j * arg)
    if kind == "DCT1":
        w = 2.0 - (j == 0) - (j == n)
        return w[None, :] * np.cos(arg)
    if kind == "DCT3":
        w = 2.0 - (j == 0)
        return w[None, :] * np.cos(arg)
    if kind == "DST1":
        return 2.0 * np.sin(arg)
    if kind == "DST3":
        w = 2.0 - (j == n)
        return w[None, :] * np.sin(arg)
    raise ValueError(kind)


def inverse_matrix(kind, n):
    """Inverse of the forward matrix (iDT(DT(G)) = G, Sec. 2.7.2)."""
    return np.linalg.inv(forward_matrix(kind, n))


def r2hc_matrix(n):
    """Real halfcomplex DFT (FFTW R2HC layout) of length n."""
    j = np.arange(n)
    M = np.zeros((n, n))
    for k in range(n // 2 + 1):
        M[k] = np.cos(2 * np.pi * j * k / n)
    for k in range(1, (n + 1) // 2):
        M[n - k] = -np.sin(2 * np.pi * j * k / n)
    return M


def _apply_matrix(M, x, axis):
    x = np.moveaxis(x, axis, -1)
    y = x @ M.T
    return np.moveaxis(y, -1, axis)


def _fast_forward(kind, x, axis, workers):
    if kind == "DFT":
        return sfft.fft(x, axis=axis, workers=workers)
    t = {"DCT1": ("dct", 1), "DCT3": ("dct", 3), "DST1": ("dst", 1), "DST3": ("dst", 3)}[kind]
    f = sfft.dct if t[0] == "dct" else sfft.dst
    return f(x, type=t[1], axis=axis, workers=workers)


def _fast_inverse(kind, X, axis, n, workers):
    # Inverse pairs (FFTW REDFT00/01/10, RODFT00/01/10 conventions): DCT-I^-1 = DCT-I/(2n),
    # DCT-III^-1 = DCT-II/(2n), DST-I^-1 = DST-I/(2n), DST-III^-1 = DST-II/(2n), DFT^-1 = ifft.
    if kind == "DFT":
        return sfft.ifft(X, axis=axis, workers=workers)
    t = {"DCT1": ("dct", 1), "DCT3": ("dct", 2), "DST1": ("dst", 1), "DST3": ("dst", 2)}[kind]
    f = sfft.dct if t[0] == "dct" else sfft.dst
    if np.iscomplexobj(X):
        return (f(X.real, type=t[1], axis=axis, workers=workers)
                + 1j * f(X.imag, type=t[1], axis=axis, workers=workers)) / (2.0 * n)
    return f(X, type=t[1], axis=axis, workers=workers) / (2.0 * n)


def dt_axis(x, axis, kind, n, inverse=False, fast=None, workers=-1):
    """Apply the forward (or inverse) transform of `kind` along `axis` of x.

    x holds the transform's own range along `axis` (node range forward,
    frequency range inverse); the length is preserved.
    """
    if fast is None:
        fast = n > DENSE_MAX
    if fast:
        if inverse:
            return _fast_inverse(kind, x, axis, n, workers)
        return _fast_forward(kind, x, axis, workers)
    M = inverse_matrix(kind, n) if inverse else forward_matrix(kind, n)
    return _apply_matrix(M, x, axis)


def dt3d_forward(g, kinds, n, fast=None):
    """3D forward DT of one node-field component (Sec. 2.7.2: x, then y, then z).

    g: array over the full stored node grid; only each axis' node range is used.
    Returns the spectral array (complex if any axis is a DFT, else real).
    """
    sl = tuple(slice(*dof_range(kinds[a], n[a])) for a in range(3))
    x = np.asarray(g, dtype=np.float64)[sl]
    for a in range(3):
        x = dt_axis(x, a, kinds[a], n[a], fast=fast)
    return x


def dt3d_inverse(X, kinds, n, node_shape, fast=None):
    """3D inverse DT back onto the node grid; dismissed nodes are set to 0."""
    x = X
    for a in (2, 1, 0):
        x = dt_axis(x, a, kinds[a], n[a], inverse=True, fast=fast)
    if np.iscomplexobj(x):
        x = x.real
    out = np.zeros(node_shape)
    sl = tuple(slice(*dof_range(kinds[a], n[a])) for a in range(3))
    out[sl] = x
    return out


def extended_field(g, left, right):
    """'Virtually' extended periodic field E of a 1D node field g (Sec. 2.4, Fig. Symmetries).

    g has n+1 node values j = 0..n.  P/P: E = g[0:n] (period n).  S/S and A/A:
    period 2n.  S/A and A/S: period 4n (reflect about node n, then about node 0).
    Symmetric: e(-j) = e(j); anti-symmetric: e(-j) = -e(j) (zero on the face).
    Returns (E, S_f).
    """
    g = np.asarray(g, dtype=np.float64)
    n = g.size - 1
    if (left, right) == ("P", "P"):
        return g[:n].copy(), 1
    sl = 1.0 if left == "S" else -1.0
    sr = 1.0 if right == "S" else -1.0
    if left == right:
        period = 2 * n
    else:
        period = 4 * n
    E = np.zeros(period)

    def val(j):
        # value of the extension at integer node j (any integer), by reflecting into [0, n]
        sign = 1.0
        j = j % period
        # fold into [0, period/2] with the left reflection (about 0)
        if j > period // 2:
            j = period - j
            sign *= sl
        # fold into [0, n] with the right reflection (about n), possibly twice for 4n periods
        while j > n:
            j = 2 * n - j
            sign *= sr
            if j < 0:
                j = -j
                sign *= sl
        return sign * g[j]

    for j in range(period):
        E[j] = val(j)
    return E, (period // n)
