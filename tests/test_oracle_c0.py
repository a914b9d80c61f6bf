"""The oracle's C0 discrete Green operator (Sec. 2.6.1, Eqs. TF_C0_behavior, FourierSGO,
FourierSGO_HEX1), pinned by its real-space definition.

* For every normal-mixed BC combination of Eq. SGO_BCs on non-periodic axes (per axis: normal
  component Dirichlet and tangential ones Neumann, or the converse), HEX1 and TETRA2,
  anisotropic voxels:
  the DCT/DST coefficients of div(C0 : grad u) computed in real space with the ghost rules
  (stencils.div) equal the symbol -(2 mu0 |xi|^2 u + lambda0 (v . u) v) on the coefficients of
  u, for random u.  A sign slip in v (one component's tau flipped) must break the identity.
* The Green operator inverts the symbol on every non-null mode.
* A fixed point preconditioned with C0 converges to the solution the B0-preconditioned one
  reaches (a different preconditioner, the same discrete problem), in fewer iterations on a
  nearly incompressible-free isotropic composite.
* Both schemes (TETRA2: Eqs. FourierSGO_TETRA2_1/2, a 2 x 2 system per frequency).
* Unsupported cases are refused: a periodic axis, BCs that are not normal-mixed.
"""

import itertools

import numpy as np
import pytest

from oracle.bc import Grid
from oracle.green import c0_green_apply, c0_symbol_apply, c0_unsupported, c0_vectors
from oracle.laws import c0_apply
from oracle.solver import Problem
from oracle.stencils import div, grad
from oracle.transforms import dt3d_forward

LAM0, MU0 = 1.3, 0.7


def _bc(choice):
    """choice[a] = 'D' (normal Dirichlet, tangential Neumann) or 'N' (the converse)."""
    other = {"D": "N", "N": "D"}
    bc = []
    for a in range(3):
        face = [choice[a] if q == a else other[choice[a]] for q in range(3)]
        bc.append([list(face), list(face)])
    return bc


def _coeffs(field, g):
    out = []
    for q in range(3):
        full = np.zeros(g.N)
        full[g.dof_slices(q)] = dt3d_forward(field[q], g.kind[q], g.n)
        out.append(full)
    return out


def _random_u(g, seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(g.node_shape)
    for q in range(3):
        u[q][~g.dof_mask(q)] = 0.0
    return u


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
@pytest.mark.parametrize("choice", list(itertools.product("DN", repeat=3)))
def test_real_space_operator_equals_the_symbol(choice, scheme):
    g = Grid((6, 5, 4), _bc(choice), h=(1.0, 0.8, 1.3))
    assert c0_unsupported(g, scheme) is None
    u = _random_u(g, 3)
    p = div(c0_apply(grad(u, g, scheme), LAM0, MU0), g, scheme)
    for q in range(3):
        p[q][~g.dof_mask(q)] = 0.0
    ph = _coeffs(p, g)
    uh = _coeffs(u, g)
    sym = c0_symbol_apply(g, LAM0, MU0, uh, scheme)
    for q in range(3):
        m = np.zeros(g.N, dtype=bool)
        m[g.dof_slices(q)] = True
        ref = np.abs(ph[q][m]).max()
        assert np.abs(sym[q][m] - ph[q][m]).max() <= 1e-12 * ref, (choice, q)
    # a planted sign slip in v (and in w for TETRA2): the identity must fail
    v, w, xx = c0_vectors(g, scheme)
    v[0] = -v[0]
    w[1] = -w[1]
    vu = sum(v[q] * uh[q] for q in range(3))
    wu = sum(w[q] * uh[q] for q in range(3))
    bad = [-(2.0 * MU0 * xx * uh[q] + LAM0 * (vu * v[q] + wu * w[q])) for q in range(3)]
    worst = max(np.abs(bad[q] - ph[q]).max() / np.abs(ph[q]).max() for q in range(3))
    assert worst > 1e-3


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
@pytest.mark.parametrize("choice", [("D", "N", "D"), ("N", "D", "N")])
def test_green_inverts_the_symbol(choice, scheme):
    g = Grid((6, 5, 4), _bc(choice), h=(1.0, 0.8, 1.3))
    uh = _coeffs(_random_u(g, 5), g)
    back = c0_green_apply(g, LAM0, MU0, c0_symbol_apply(g, LAM0, MU0, uh, scheme), scheme)
    v, w, xx = c0_vectors(g, scheme)
    for q in range(3):
        m = np.zeros(g.N, dtype=bool)
        m[g.dof_slices(q)] = True
        m &= xx > 0
        assert np.abs(back[q][m] - uh[q][m]).max() <= 1e-12 * np.abs(uh[q][m]).max()


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_c0_and_b0_fixed_points_agree(scheme):
    import synthetic as syn
    from synthetic.workloads import ISO_ELASTIC, Material, Workload

    n = (12, 10, 8)
    ph = syn.random_spheres(n, 0.2, 1.5, 2.5, 11)
    E, nu = 1.0, 0.3
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    mats = [Material(ISO_ELASTIC, (lam, mu)), Material(ISO_ELASTIC, (5 * lam, 5 * mu))]
    A = np.zeros((3, 3))
    A[0, 0] = 1e-3
    out = {}
    for green in ("B0", "C0"):
        wl = Workload("c0_vs_b0", n, ph, mats, _bc(("D", "N", "N")), scheme=scheme, green=green,
                      lambda0=3 * lam, mu0=3 * mu, tol=1e-11, A=A, max_iter=2000)
        pr = Problem(wl)
        _, rep = pr.solve_step()
        assert rep.converged, green
        out[green] = (pr.last["P"], rep.iterations)
    P_b, it_b = out["B0"]
    P_c, it_c = out["C0"]
    assert np.linalg.norm(P_c - P_b) <= 1e-8 * np.linalg.norm(P_b)
    assert it_c <= it_b, (it_c, it_b)


def test_unsupported_cases_are_refused():
    bc = _bc(("D", "N", "D"))
    bc[2] = [["P"] * 3, ["P"] * 3]
    assert c0_unsupported(Grid((6, 5, 4), bc), "HEX1") is not None
    bc = _bc(("D", "N", "D"))
    bc[1] = [["D"] * 3, ["D"] * 3]  # all components Dirichlet on y: not normal-mixed
    assert c0_unsupported(Grid((6, 5, 4), bc), "HEX1") is not None
