"""Oracle fixed point (Algorithm 1) pinned by exact solutions.

T5  law = preconditioner (B0): one Green application solves the step exactly
T6  laminate closed forms (layers normal to x; layers normal to y with equal nu)
T7  a direct sparse solve of the same discrete system (strains and stresses)
    Anderson: constrained least-squares optimality and the skip rule
"""

import numpy as np
import pytest

import synthetic as syn
from oracle import anderson, direct
from oracle.solver import Problem
from oracle.stencils import grad
from synthetic.workloads import B0_LINEAR, CUBIC_ELASTIC, Material, Workload, axis_bc


def _strain(G):
    return 0.5 * (G + np.swapaxes(G, 1, 2))


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
@pytest.mark.parametrize("bc", [axis_bc("D", "N", "P"), axis_bc("N", "D", "D"),
                                [[["D", "N", "N"], ["D", "N", "N"]], [["N", "D", "N"], ["N", "D", "N"]],
                                 [["P"] * 3] * 2]])
def test_one_iteration_exact_when_law_is_the_preconditioner(scheme, bc):
    n = (6, 5, 4)
    A = np.array([[1e-3, 2e-4, 0.0], [0.0, -3e-4, 1e-4], [5e-5, 0.0, 0.0]])
    wl = Workload("b0", n, np.zeros(n, np.uint16), [Material(B0_LINEAR, (2.0, 1.5))], bc,
                  scheme=scheme, lambda0=2.0, mu0=1.5, tol=1e-13, A=A, max_iter=5)
    pr = Problem(wl)
    # u* must not depend on a periodic coordinate
    for a in range(3):
        if pr.grid.periodic[a]:
            wl.A[:, a] = 0.0
    _, rep = pr.solve_step(anderson=False)
    assert rep.err[0] > 1e-6
    assert rep.iterations == 1 and rep.converged, rep.err


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_x_laminate_closed_form(scheme):
    wl = syn.x_laminate(scheme=scheme)
    pr = Problem(wl)
    _, rep = pr.solve_step()
    assert rep.converged
    lam = np.array([m.params[0] for m in wl.materials])
    mu = np.array([m.params[1] for m in wl.materials])
    M = (lam + 2 * mu)[wl.phase[:, 0, 0]]
    s11 = 1e-3 / np.mean(1.0 / M)
    P = pr.last["P"]
    assert np.abs(P[:, 0, 0] - s11).max() < 1e-9 * s11
    for i, q in [(0, 1), (0, 2), (1, 2), (1, 0), (2, 0), (2, 1)]:
        assert np.abs(P[:, i, q]).max() < 1e-9 * s11
    # lateral stresses lambda * eps_11 in each layer
    eps = s11 / M
    assert np.allclose(P[0, 1, 1], (lam[wl.phase[:, 0, 0]] * eps)[:, None, None], rtol=1e-8)


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_y_laminate_closed_form(scheme):
    wl = syn.y_laminate(scheme=scheme)
    pr = Problem(wl)
    _, rep = pr.solve_step()
    assert rep.converged
    E = np.array([1.0, 5.0])
    nu = 0.25
    s11 = (E / (1 - nu ** 2) * 1e-3)[wl.phase[0, :, 0]]
    P = pr.last["P"]
    assert np.abs(P[0, 0, 0] - s11[None, :, None]).max() < 1e-9 * s11.max()
    assert np.abs(P[0, 1, 1]).max() < 1e-9 * s11.max()
    assert np.abs(P[0, 2, 2] - nu * P[0, 0, 0]).max() < 1e-9 * s11.max()


BCS_T7 = [axis_bc("D", "D", "P"), axis_bc("D", "N", "N"), axis_bc("D", "N", "P"),
          [[["D", "N", "D"], ["N", "D", "D"]], [["D", "D", "N"], ["N", "N", "D"]], [["P"] * 3, ["P"] * 3]]]


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
@pytest.mark.parametrize("bci", range(len(BCS_T7)))
def test_fixed_point_matches_direct_sparse_solve(scheme, bci):
    bc = BCS_T7[bci]
    n = (7, 6, 5)
    ph, _ = syn.voronoi(n, 4, 7)
    quats = syn.shoemake_quaternions(4, 8)
    mats = [Material(CUBIC_ELASTIC, (168.0, 121.0, 75.0), tuple(q)) for q in quats]
    A = np.zeros((3, 3))
    A[0, 0] = 1e-3
    A[1, 0] = 4e-4
    wl = Workload("t7", n, ph, mats, bc, scheme=scheme, lambda0=121.0, mu0=49.25,
                  tol=1e-12, A=A, max_iter=3000)
    pr = Problem(wl)
    uf, rep = pr.solve_step()
    assert rep.converged
    ud = direct.solve(wl, pr.grad_ustar())
    e1 = _strain(grad(uf, pr.grid, scheme))
    e2 = _strain(grad(ud, pr.grid, scheme))
    assert np.abs(e1 - e2).max() < 1e-9 * np.abs(e2).max()


def test_anderson_coefficients_are_the_constrained_minimiser():
    rng = np.random.default_rng(4)
    fs = [rng.standard_normal(50) for _ in range(4)]
    c = anderson.coefficients(fs)
    assert abs(c.sum() - 1.0) < 1e-14
    best = np.linalg.norm(sum(ci * f for ci, f in zip(c, fs)))
    for _ in range(200):
        d = rng.standard_normal(4)
        d -= d.mean()
        trial = c + 1e-3 * d
        assert np.linalg.norm(sum(ci * f for ci, f in zip(trial, fs))) >= best - 1e-12


def test_anderson_recovers_an_exact_cancellation_and_skips_degenerate_history():
    rng = np.random.default_rng(9)
    a, b = rng.standard_normal(30), rng.standard_normal(30)
    fs = [a, b, a + b, 2 * a - b + rng.standard_normal(30)]
    c = anderson.coefficients(fs)
    assert np.linalg.norm(sum(ci * f for ci, f in zip(c, fs))) < np.linalg.norm(fs[-1])
    same = [a, a, a, a]
    assert anderson.coefficients(same) is None
    assert anderson.accelerate_now(5, 3, 4, 4) and not anderson.accelerate_now(4, 3, 4, 4)
    assert not anderson.accelerate_now(2, 3, 2, 4)


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_bending_load_matches_direct_sparse_solve(scheme):
    """T7 with the bilinear u* of a bending load (x faces clamped, y and z traction-free)."""
    n = (8, 6, 5)
    ph = syn.random_spheres(n, 0.3, 1.0, 2.0, 11)
    mats = [Material(0, syn.iso_lame(1.0, 0.3)), Material(0, syn.iso_lame(4.0, 0.25))]
    A, b, Q = syn.bending_load(n, (1.0, 1.0, 1.0), 0.01)
    wl = Workload("t7b", n, ph, mats, axis_bc("D", "N", "N"), scheme=scheme, lambda0=1.6, mu0=1.0,
                  tol=1e-12, A=A, b=b, Q=Q, max_iter=3000)
    pr = Problem(wl)
    uf, rep = pr.solve_step()
    assert rep.converged
    ud = direct.solve(wl, pr.grad_ustar())
    e1 = _strain(grad(uf, pr.grid, scheme))
    e2 = _strain(grad(ud, pr.grid, scheme))
    assert np.abs(e1 - e2).max() < 1e-9 * np.abs(e2).max()
    # a bending moment, not a net force: the mean axial stress is far below its extreme values
    P = pr.last["P"]
    assert abs(P[:, 0, 0].mean()) < 0.2 * np.abs(P[:, 0, 0]).max()


def _uniaxial_j2_history(strains, E, sy, H):
    """1D plasticity with linear isotropic hardening (the uniaxial-stress form of J2):
    sigma = E (eps - eps_p), |sigma| <= sy + H p, backward-Euler return at each step."""
    ep, p, out = 0.0, 0.0, []
    for eps in strains:
        trial = E * (eps - ep)
        f = abs(trial) - (sy + H * p)
        if f > 0.0:
            dp = f / (E + H)
            ep += dp * np.sign(trial)
            p += dp
        out.append((E * (eps - ep), p))
    return out


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_j2_bar_loading_and_unloading_follow_the_uniaxial_closed_form(scheme):
    """A homogeneous J2 bar, normal-only Dirichlet on x and traction-free elsewhere, is in
    uniaxial stress at every step; loading past yield and unloading checks the committed
    state (eps^p, p) carried from step to step (Algorithm 1, step commit)."""
    E, nu, sy, H = 200.0, 0.3, 0.3, 2.0
    lam, mu = syn.iso_lame(E, nu)
    n = (5, 4, 3)
    bc = axis_bc("D", "N", "N")
    bc[0] = [["D", "N", "N"], ["D", "N", "N"]]
    wl = Workload("j2bar", n, np.zeros(n, np.uint16), [Material(2, (lam, mu, sy, H))], bc,
                  scheme=scheme, lambda0=lam, mu0=mu, tol=1e-11, max_iter=3000)
    pr = Problem(wl)
    strains = [1e-3, 2e-3, 3e-3, 2.5e-3, 1e-3, 3.5e-3]
    expect = _uniaxial_j2_history(strains, E, sy, H)
    for eps, (s11, p) in zip(strains, expect):
        A = np.zeros((3, 3))
        A[0, 0] = eps
        _, rep = pr.solve_step(A=A)
        assert rep.converged, rep.err[-3:]
        P = pr.last["P"]
        assert np.abs(P[:, 0, 0] - s11).max() < 1e-8 * abs(s11), (eps, P[:, 0, 0].mean(), s11)
        assert np.abs(P[:, 1, 1]).max() < 1e-8 * abs(s11)
        assert np.abs(pr.state["p"] - p).max() < 1e-8 * max(p, 1e-3)
    assert expect[2][1] > 0 and expect[3][1] == expect[2][1]  # yielded, then unloaded elastically
