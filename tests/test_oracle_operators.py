"""Oracle stencils, ghost rules and Green operator.

T3  real-space div(B0 : grad u) vs the DT-diagonal symbol, every BC combination
    (the cross-validation of Sec. 2.7.3), HEX1 and TETRA2, plus random
    per-component BCs with anisotropic voxels
T4  adjointness: div = -grad^T with nodal weights (Remark 1)
    linear exactness of the stencils; the null-denominator pattern of the Green operator
"""

import itertools

import numpy as np
import pytest

from oracle.bc import KIND_OF_PAIR, Grid, half_angles
from oracle.green import green_factor, operator_symbol
from oracle.laws import b0_apply
from oracle.stencils import div, grad, grad_full, node_weights
from oracle.transforms import dt3d_forward, dt3d_inverse

BC_OF_SYM = {"P": "P", "S": "N", "A": "D"}
PAIRS = list(KIND_OF_PAIR.keys())


def _masked_random(g, rng):
    u = rng.standard_normal(g.node_shape)
    for q in range(3):
        u[q][~g.dof_mask(q)] = 0.0
    return u


def _fourier_operator(u, g, scheme, lam0, mu0):
    out = np.zeros_like(u)
    for q in range(3):
        spec = dt3d_forward(u[q], g.kind[q], g.n)
        out[q] = dt3d_inverse(spec * operator_symbol(g, q, scheme, lam0, mu0), g.kind[q], g.n, g.N)
    return out


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
@pytest.mark.parametrize("lam0,mu0", [(1.7, 0.9), (0.0, 1.0), (3.0, 0.0)])
def test_cross_validation_all_axis_pairs(scheme, lam0, mu0):
    rng = np.random.default_rng(11)
    worst = 0.0
    for tri in itertools.product(PAIRS, repeat=3):
        bc = [[[BC_OF_SYM[tri[a][f]]] * 3 for f in range(2)] for a in range(3)]
        g = Grid((5, 6, 4), bc)
        u = _masked_random(g, rng)
        real = div(b0_apply(grad(u, g, scheme), lam0, mu0), g, scheme)
        four = _fourier_operator(u, g, scheme, lam0, mu0)
        for q in range(3):
            m = g.dof_mask(q)
            den = np.sum(real[q][m] ** 2)
            if den == 0.0:
                continue
            worst = max(worst, np.sum((real[q][m] - four[q][m]) ** 2) / den)
    assert worst < 1e-26


def test_cross_validation_mixed_components_anisotropic():
    rng = np.random.default_rng(12)
    for trial in range(120):
        bc = []
        for a in range(3):
            if rng.random() < 0.25:
                bc.append([["P"] * 3, ["P"] * 3])
            else:
                bc.append([[str(rng.choice(["D", "N"])) for _ in range(3)] for _ in range(2)])
        n = tuple(int(v) for v in rng.integers(3, 7, size=3))
        h = tuple(rng.uniform(0.5, 2.0, size=3))
        g = Grid(n, bc, h)
        scheme = "HEX1" if trial % 2 else "TETRA2"
        u = _masked_random(g, rng)
        real = div(b0_apply(grad(u, g, scheme), 1.3, 0.7), g, scheme)
        four = _fourier_operator(u, g, scheme, 1.3, 0.7)
        for q in range(3):
            m = g.dof_mask(q)
            assert np.sum((real[q][m] - four[q][m]) ** 2) <= 1e-26 * np.sum(real[q][m] ** 2)


def test_cross_validation_detects_a_planted_ghost_sign_error(monkeypatch):
    """A wrong sign in the ghost rule must break the cross-validation."""
    import oracle.stencils as st

    orig = st.ghost_extend

    def broken(S, grid, scheme):
        E = orig(S, grid, scheme)
        E[:, 0, 1, 0] *= -1.0  # flip the left-x ghost of S_12
        return E

    monkeypatch.setattr(st, "ghost_extend", broken)
    rng = np.random.default_rng(3)
    g = Grid((5, 5, 4), [[["D"] * 3, ["N"] * 3], [["N"] * 3, ["N"] * 3], [["P"] * 3, ["P"] * 3]])
    u = _masked_random(g, rng)
    real = st.div(b0_apply(st.grad(u, g, "HEX1"), 1.0, 1.0), g, "HEX1")
    four = _fourier_operator(u, g, "HEX1", 1.0, 1.0)
    assert np.abs(real - four).max() > 1e-3


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_gradient_exact_for_affine_fields(scheme):
    g = Grid((4, 5, 3), [[["D"] * 3] * 2, [["N"] * 3] * 2, [["D"] * 3] * 2], h=(0.5, 1.5, 2.0))
    A = np.arange(9.0).reshape(3, 3) - 4.0
    x = [np.arange(g.n[a] + 1) * g.h[a] for a in range(3)]
    X = np.meshgrid(*x, indexing="ij")
    uf = np.stack([A[q, 0] * X[0] + A[q, 1] * X[1] + A[q, 2] * X[2] + q for q in range(3)])
    G = grad_full(uf, g, scheme)
    for r in range(G.shape[0]):
        for i in range(3):
            for q in range(3):
                assert np.allclose(G[r, i, q], A[q, i], atol=1e-12)


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_divergence_is_minus_weighted_adjoint_of_gradient(scheme):
    """<W div S, v> = -<S, grad v> / n_ppv for S with the symmetries of grad u^f."""
    rng = np.random.default_rng(5)
    for bc in ([[["P"] * 3] * 2] * 3,
               [[["D", "N", "D"], ["N", "N", "D"]], [["N"] * 3, ["D"] * 3], [["P"] * 3] * 2],
               [[["D"] * 3] * 2, [["N"] * 3] * 2, [["N", "D", "N"], ["D", "N", "N"]]]):
        g = Grid((5, 4, 6), bc, h=(1.0, 0.7, 1.3))
        npp = 1 if scheme == "HEX1" else 2
        S = rng.standard_normal((npp, 3, 3) + g.n)
        v = _masked_random(g, rng)
        lhs = np.sum(node_weights(g)[None] * div(S, g, scheme) * v)
        rhs = -np.sum(S * grad(v, g, scheme)) / npp
        assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(rhs))


def test_green_null_pattern():
    """HEX1 nulls: all-zero frequencies or >= 2 axes at pi; TETRA2: all-zero or all-pi."""
    g = Grid((4, 4, 4), [[["P"] * 3] * 2, [["N"] * 3] * 2, [["P"] * 3] * 2])
    kinds = g.kind[0]
    flags = []
    for a in range(3):
        s, c = half_angles(kinds[a], g.n[a])
        flags.append((s == 0.0, c == 0.0))
    for scheme in ("HEX1", "TETRA2"):
        f = green_factor(g, 0, scheme, 1.0, 1.0)
        for k in itertools.product(*[range(f.shape[a]) for a in range(3)]):
            zero = [flags[a][0][k[a]] for a in range(3)]
            pi = [flags[a][1][k[a]] for a in range(3)]
            if scheme == "HEX1":
                null = all(zero) or sum(pi) >= 2
            else:
                null = all(zero) or all(pi)
            assert (f[k] == 0.0) == null, (scheme, k)


def test_gradient_of_quadratic_load_fields_closed_form():
    """The monomials of a quadratic u* on the node grid.  Worked out by hand from the four
    (TETRA2, Eqs. D1T1T2G-D3T1T2G) or eight (HEX1, Eqs. D1HG-D3HG) corners:
    D_i (x_a^2) = 2 x_a delta_ia at the voxel centre for both schemes;
    D_i (x_a x_b) = x_b delta_ia + x_a delta_ib, plus, on the third axis c, 0 for HEX1 and
    -h_a h_b / (2 h_c) on T1, +h_a h_b / (2 h_c) on T2."""
    h = (0.7, 1.3, 0.9)
    n = (5, 4, 3)
    g = Grid(n, [[["P"] * 3] * 2] * 3, h)
    X = np.meshgrid(*[np.arange(n[a] + 1) * h[a] for a in range(3)], indexing="ij")
    Xc = np.meshgrid(*[(np.arange(n[a]) + 0.5) * h[a] for a in range(3)], indexing="ij")
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    for a, b in pairs:
        u = np.zeros((3,) + tuple(v + 1 for v in n))
        u[2] = X[a] * X[b]  # component q = 2 only
        for scheme in ("HEX1", "TETRA2"):
            G = grad_full(u, g, scheme)
            assert np.abs(G[:, :, :2]).max() == 0.0
            for r in range(G.shape[0]):
                for i in range(3):
                    expect = (Xc[b] if i == a else 0.0) + (Xc[a] if i == b else 0.0)
                    if a != b and i not in (a, b) and scheme == "TETRA2":
                        expect = expect + (-1.0 if r == 0 else 1.0) * h[a] * h[b] / (2 * h[i])
                    assert np.allclose(G[r, i, 2], expect, rtol=0, atol=1e-12), (a, b, scheme, r, i)
