"""Oracle transforms pinned against Table 1 independently of the Table-1 transcription.

T1  dense Table-1 matrices vs the scipy fast path (both directions)
T1b DT(G) vs the explicit DFT of the virtually extended field (alpha, S_f, index map)
T2  iDT(DT(G)) = G for every per-axis transform triple (Sec. 2.7.2 validation)
"""

import itertools
import os

import numpy as np
import pytest

from oracle.bc import KIND_OF_PAIR, KINDS, dof_range, frequencies, n_freq
from oracle.transforms import (dt3d_forward, dt3d_inverse, dt_axis, extended_field,
                               forward_matrix, inverse_matrix, r2hc_matrix)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_links.txt")
SIZES = [2, 3, 4, 5, 6, 7, 8, 9, 16, 31, 32, 33, 48]


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        l, r, kind, sf, are, aim, idx = line.split()
        rows.append((l, r, kind, int(sf), complex(float(are), float(aim)), idx))
    return rows


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", SIZES + [64, 96])
def test_fast_path_matches_table1_matrices(kind, n):
    rng = np.random.default_rng(n)
    L = n_freq(kind, n)
    x = rng.standard_normal((3, L))
    dense = dt_axis(x, 1, kind, n, fast=False)
    fast = dt_axis(x, 1, kind, n, fast=True)
    assert np.allclose(dense, fast, rtol=0, atol=1e-11 * max(1.0, np.abs(dense).max()))
    back_dense = dt_axis(dense, 1, kind, n, inverse=True, fast=False)
    back_fast = dt_axis(dense, 1, kind, n, inverse=True, fast=True)
    assert np.allclose(back_dense, x, atol=1e-11)
    assert np.allclose(back_fast, x, atol=1e-11)


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[2])
@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8, 12])
def test_dt_equals_alpha_times_dft_of_extension(row, n):
    left, right, kind, sf, alpha, idx = row
    assert KIND_OF_PAIR[(left, right)] == kind
    rng = np.random.default_rng(100 + n)
    g = rng.standard_normal(n + 1)
    if left == "A":
        g[0] = 0.0
    if right == "A":
        g[n] = 0.0
    if kind == "DFT":
        g[n] = g[0]
    E, Sf = extended_field(g, left, right)
    assert Sf == sf
    Ehat = np.fft.fft(E)
    lo, hi = dof_range(kind, n)
    Gt = forward_matrix(kind, n) @ g[lo:hi]
    for k in range(Gt.size):
        b = {"k": k, "k+1": k + 1, "2k+1": 2 * k + 1}[idx]
        assert abs(Ehat[b] - alpha * Gt[k]) <= 1e-11 * max(1.0, np.abs(Ehat).max())
    # the fundamental frequency is the DFT frequency of that bin of E
    xi, _, _ = frequencies(kind, n)
    for k in range(Gt.size):
        b = {"k": k, "k+1": k + 1, "2k+1": 2 * k + 1}[idx]
        assert abs(xi[k] - 2 * np.pi * b / (sf * n)) < 1e-14


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [3, 4, 7, 8])
def test_inverse_matrix_is_the_fftw_inverse_pair(kind, n):
    """DCT-I^-1 = DCT-I/2n, DCT-III^-1 = DCT-II/2n, DST-I^-1 = DST-I/2n, DST-III^-1 = DST-II/2n."""
    Minv = inverse_matrix(kind, n)
    L = n_freq(kind, n)
    k = np.arange(L)
    if kind == "DFT":
        ref = np.exp(2j * np.pi * np.outer(np.arange(n), k) / n) / n
    elif kind == "DCT1":
        j = np.arange(n + 1)
        w = 2.0 - (k == 0) - (k == n)
        ref = (w[None, :] * np.cos(np.pi * np.outer(j, k) / n)) / (2 * n)
    elif kind == "DCT3":
        j = np.arange(n)
        ref = 2 * np.cos(np.pi * np.outer(j, k + 0.5) / n) / (2 * n)
    elif kind == "DST1":
        j = np.arange(1, n)
        ref = 2 * np.sin(np.pi * np.outer(j, k + 1) / n) / (2 * n)
    else:
        j = np.arange(1, n + 1)
        ref = 2 * np.sin(np.pi * np.outer(j, k + 0.5) / n) / (2 * n)
    assert np.allclose(Minv, ref, atol=1e-12)


TRIPLES = list(itertools.product(KINDS, repeat=3))


@pytest.mark.parametrize("n", [(5, 4, 6), (8, 9, 7)])
def test_round_trip_every_triple(n):
    rng = np.random.default_rng(7)
    for kinds in TRIPLES:
        N = tuple(n[a] if kinds[a] == "DFT" else n[a] + 1 for a in range(3))
        g = rng.standard_normal(N)
        sl = tuple(slice(*dof_range(kinds[a], n[a])) for a in range(3))
        mask = np.zeros(N, dtype=bool)
        mask[sl] = True
        g[~mask] = 0.0
        back = dt3d_inverse(dt3d_forward(g, kinds, n), kinds, n, N)
        assert np.abs(back - g).max() < 1e-12, kinds


@pytest.mark.parametrize("n", [2, 3, 6, 7, 16])
def test_r2hc_matrix_packs_the_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    X = np.fft.fft(x)
    y = r2hc_matrix(n) @ x
    for k in range(n // 2 + 1):
        assert abs(y[k] - X[k].real) < 1e-12
    for k in range(1, (n + 1) // 2):
        assert abs(y[n - k] - X[k].imag) < 1e-12
