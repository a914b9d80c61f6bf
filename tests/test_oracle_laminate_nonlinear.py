"""Pins of the oracle's full-field solve for nonlinear laws against an independent construction.

A laminate of two materials (layers normal to x, three voxels each, Dirichlet x faces, periodic
y and z) under an affine displacement u* = A x that depends on x only has a displacement
fluctuation depending on x only, piecewise linear with kinks at the interfaces: the HEX1 and
TETRA2 gradients are then exact in every voxel, the gradient of each layer is
G_L = G* + e1 (x) g_L with the zero-mean condition n_A g_A + n_B g_B = 0 (u^f vanishes on both
x faces), and the divergence vanishes everywhere iff the traction on the interface planes is
continuous, S_A[0, :] = S_B[0, :] (Eq. GeneralBCtobesolved with the stencils of Sec. 2.5).  The
tests solve those three equations for g_A by their own Newton iteration, with the oracle's
pointwise law of each layer (pinned separately: single-slip recursion for crystal plasticity,
closed forms for the others) from the virgin state, and compare with Algorithm 1 run by the
oracle on the full grid: FCC crystal plasticity past yield (power-law slip with Voce hardening,
the crystal law of Sec. 3.4 as the oracle states it), small-strain J2 past yield on both
stencils, logarithmic J2 past yield (Sec. 3.2), Neo-Hookean (Appendix B) and cubic
St-Venant-Kirchhoff at 5-10 % strain."""

import numpy as np
import pytest

import synthetic as syn
from oracle.finite import cp_fcc
from oracle.solver import Problem
from synthetic.workloads import CP_FCC, CP_FCC_PARAMS, Material, Workload, axis_bc


def _layer_law(G, mat):
    """S (3, 3) and the cumulated slip at one point of a virgin crystal."""
    Fp = np.eye(3).reshape(1, 3, 3, 1)
    S, _, gam = cp_fcc(G.reshape(1, 3, 3, 1), mat.params, mat.quat, Fp, np.zeros((1, 1)))
    return S[0, :, :, 0], float(gam.ravel()[0])


def _layer_stress(G, mat):
    return _layer_law(G, mat)[0]


def test_cp_laminate_matches_the_traction_continuity_solution():
    n = (12, 2, 2)
    phase = syn.laminate(n, 0, 3)
    quats = syn.shoemake_quaternions(2, 11)
    mats = [Material(CP_FCC, CP_FCC_PARAMS, tuple(q)) for q in quats]
    A = np.zeros((3, 3))
    A[0, 0], A[1, 0], A[2, 0] = 1.5e-3, 4e-3, -2e-3  # u*_q = A[q][0] x: stretch and two shears
    C11, C12, C44 = CP_FCC_PARAMS[:3]
    wl = Workload(name="cp_laminate", n=n, phase=phase, materials=mats, bc=axis_bc("D", "P", "P"),
                  scheme="HEX1", green="B0", lambda0=C12, mu0=0.5 * (C44 + 0.5 * (C11 - C12)),
                  tol=1e-10, A=A, max_iter=3000)
    pr = Problem(wl)
    _, rep = pr.solve_step()
    assert rep.converged

    # the three-equation laminate problem, solved independently
    Gs = np.zeros((3, 3))
    Gs[0, :] = A[:, 0]  # G*_iq = d u*_q / d x_i
    nA = int(np.sum(phase[:, 0, 0] == 0))
    nB = n[0] - nA

    def layers(g):
        GA, GB = Gs.copy(), Gs.copy()
        GA[0, :] += g
        GB[0, :] -= (nA / nB) * g
        return GA, GB

    def resid(g):
        GA, GB = layers(g)
        return _layer_stress(GA, mats[0])[0, :] - _layer_stress(GB, mats[1])[0, :]

    g = np.zeros(3)
    for _ in range(50):
        r = resid(g)
        if np.linalg.norm(r) < 1e-13:
            break
        J = np.zeros((3, 3))
        for k in range(3):
            dg = np.zeros(3)
            dg[k] = 1e-7
            J[:, k] = (resid(g + dg) - resid(g - dg)) / 2e-7
        g = g - np.linalg.solve(J, r)
    assert np.linalg.norm(resid(g)) < 1e-12
    GA, GB = layers(g)
    (SA, gA), (SB, gB) = _layer_law(GA, mats[0]), _layer_law(GB, mats[1])
    # past yield in both crystals: cumulated slip of several times the elastic limit
    assert min(gA, gB) > 1e-3, (gA, gB)

    G = pr.last["G"][0]  # (3, 3, n1, n2, n3), HEX1: one point per voxel
    P = pr.last["P"][0]
    for ph, (GL, SL) in enumerate([(GA, SA), (GB, SB)]):
        sel = phase == ph
        Gv = G[:, :, sel]
        Sv = P[:, :, sel]
        assert np.abs(Gv - GL[:, :, None]).max() <= 1e-7 * np.abs(GL).max()
        assert np.abs(Sv - SL[:, :, None]).max() <= 1e-6 * np.abs(SL).max()


# The same construction for the other nonlinear laws: small-strain J2 with hardening (both
# stencils), logarithmic J2, Neo-Hookean and cubic St-Venant-Kirchhoff, each on a laminate of
# two materials under an x-only affine load; the pointwise law of each layer is the oracle's
# (`oracle.laws.stress` at one point, from the virgin state), the equilibrium is the test's own.
from oracle.finite import log_j2  # noqa: E402
from oracle.laws import j2_return, stress  # noqa: E402
from synthetic.workloads import J2_LINHARD, LOG_J2, NEO_HOOKE, SVK_CUBIC, iso_lame  # noqa: E402


def _laminate_case(name):
    lam, mu = iso_lame(200.0, 0.3)
    if name == "j2":
        mats = [Material(J2_LINHARD, (lam, mu, 0.15, 1.0)), Material(J2_LINHARD, (lam, mu, 0.3, 2.0))]
        a = (3e-3, 2e-3, -1e-3)
    elif name == "log_j2":
        mats = [Material(LOG_J2, (lam, mu, 0.1)), Material(LOG_J2, (0.5 * lam, 0.5 * mu, 0.2))]
        a = (3e-3, 2.5e-3, -1e-3)
    elif name == "neo_hooke":
        mats = [Material(NEO_HOOKE, (1.0, 3.0)), Material(NEO_HOOKE, (4.0, 10.0))]
        a = (0.1, 0.05, -0.03)
    else:
        q = syn.shoemake_quaternions(2, 13)
        mats = [Material(SVK_CUBIC, (168.0, 121.0, 75.0), tuple(v)) for v in q]
        a = (0.05, 0.03, -0.02)
    return mats, np.array(a)


def _point_stress(G, mat):
    P, _ = stress(G.reshape(1, 3, 3, 1, 1, 1), [mat], [np.array([0])])
    return P.reshape(3, 3)


@pytest.mark.parametrize("name,scheme", [("j2", "HEX1"), ("j2", "TETRA2"), ("log_j2", "HEX1"),
                                         ("neo_hooke", "HEX1"), ("svk", "TETRA2")])
def test_laminate_solve_matches_the_traction_continuity_solution(name, scheme):
    n = (12, 2, 2)
    phase = syn.laminate(n, 0, 3)
    mats, a = _laminate_case(name)
    A = np.zeros((3, 3))
    A[:, 0] = a
    lams = [m.params[0] for m in mats if m.law != NEO_HOOKE] or [2.0 * m.params[1] for m in mats]
    mus = [m.params[1] for m in mats if m.law != NEO_HOOKE] or [m.params[0] for m in mats]
    if mats[0].law == SVK_CUBIC:
        lams, mus = [121.0], [0.5 * (75.0 + 0.5 * (168.0 - 121.0))]
    wl = Workload(name="laminate_" + name, n=n, phase=phase, materials=mats, bc=axis_bc("D", "P", "P"),
                  scheme=scheme, green="B0", lambda0=max(lams), mu0=max(mus), tol=1e-11, A=A, max_iter=3000)
    pr = Problem(wl)
    _, rep = pr.solve_step()
    assert rep.converged

    Gs = np.zeros((3, 3))
    Gs[0, :] = a
    nA = int(np.sum(phase[:, 0, 0] == 0))
    nB = n[0] - nA

    def layers(g):
        GA, GB = Gs.copy(), Gs.copy()
        GA[0, :] += g
        GB[0, :] -= (nA / nB) * g
        return GA, GB

    def resid(g):
        GA, GB = layers(g)
        return _point_stress(GA, mats[0])[0, :] - _point_stress(GB, mats[1])[0, :]

    g = np.zeros(3)
    scale = np.abs(_point_stress(Gs, mats[0])).max()
    for _ in range(60):
        r = resid(g)
        if np.linalg.norm(r) < 1e-14 * scale:
            break
        J = np.zeros((3, 3))
        h = 1e-7 * max(1.0, np.abs(a).max())
        for k in range(3):
            dg = np.zeros(3)
            dg[k] = h
            J[:, k] = (resid(g + dg) - resid(g - dg)) / (2 * h)
        g = g - np.linalg.solve(J, r)
    assert np.linalg.norm(resid(g)) < 1e-12 * scale
    GA, GB = layers(g)
    if name == "j2":  # both layers past yield
        for GL, m in ((GA, mats[0]), (GB, mats[1])):
            eps = 0.5 * (GL + GL.T)
            _, _, p = j2_return(eps.reshape(1, 3, 3, 1), np.zeros((1, 3, 3, 1)), np.zeros((1, 1)), *m.params[:4])
            assert p.ravel()[0] > 1e-4
    if name == "log_j2":
        for GL, m in ((GA, mats[0]), (GB, mats[1])):
            _, _, pl = log_j2(GL.reshape(1, 3, 3, 1), m.params, np.zeros((1, 3, 3, 1)), np.zeros((1, 1)))
            assert pl.ravel()[0] > 1e-4

    G = pr.last["G"]  # (npp, 3, 3, n1, n2, n3)
    P = pr.last["P"]
    for ph, GL in enumerate((GA, GB)):
        SL = _point_stress(GL, mats[ph])
        sel = phase == ph
        for r in range(G.shape[0]):
            assert np.abs(G[r][:, :, sel] - GL[:, :, None]).max() <= 1e-7 * np.abs(GL).max()
            assert np.abs(P[r][:, :, sel] - SL[:, :, None]).max() <= 1e-6 * np.abs(SL).max()


def _virgin_state(law):
    assert law == J2_LINHARD
    return {"ep": np.zeros((1, 3, 3, 1, 1, 1)), "p": np.zeros((1, 1, 1, 1))}


def _point_law(G, mat, st):
    P, new = stress(G.reshape(1, 3, 3, 1, 1, 1), [mat], [np.array([0])], st)
    return P.reshape(3, 3), new


@pytest.mark.parametrize("name", ["j2"])
def test_laminate_two_steps_carry_the_committed_state(name):
    """Load past yield, then reverse part of the load: the second step's fields are the
    traction-continuity solution from each layer's state committed at the end of the first
    (J2 with hardening; a reversed crystal-plasticity increment takes the oracle minutes)."""
    n = (12, 2, 2)
    phase = syn.laminate(n, 0, 3)
    lam, mu = iso_lame(200.0, 0.3)
    mats = [Material(J2_LINHARD, (lam, mu, 0.15, 1.0)), Material(J2_LINHARD, (lam, mu, 0.3, 2.0))]
    loads = [np.array([3e-3, 2e-3, -1e-3]), np.array([1e-3, -1e-3, 0.5e-3])]
    lam0, mu0 = lam, mu
    A = np.zeros((3, 3))
    A[:, 0] = loads[0]
    wl = Workload(name="laminate2_" + name, n=n, phase=phase, materials=mats, bc=axis_bc("D", "P", "P"),
                  scheme="HEX1", green="B0", lambda0=lam0, mu0=mu0, tol=1e-11, A=A, max_iter=3000)
    pr = Problem(wl)
    nA = int(np.sum(phase[:, 0, 0] == 0))
    nB = n[0] - nA
    states = [_virgin_state(m.law) for m in mats]
    for step, a in enumerate(loads):
        A = np.zeros((3, 3))
        A[:, 0] = a
        _, rep = pr.solve_step(A=A)
        assert rep.converged, step
        Gs = np.zeros((3, 3))
        Gs[0, :] = a

        def layers(g):
            GA, GB = Gs.copy(), Gs.copy()
            GA[0, :] += g
            GB[0, :] -= (nA / nB) * g
            return GA, GB

        def resid(g):
            GA, GB = layers(g)
            return _point_law(GA, mats[0], states[0])[0][0, :] - _point_law(GB, mats[1], states[1])[0][0, :]

        g = np.zeros(3)
        scale = np.abs(_point_law(Gs, mats[0], states[0])[0]).max()
        for _ in range(60):
            r = resid(g)
            if np.linalg.norm(r) < 1e-14 * scale:
                break
            J = np.zeros((3, 3))
            for k in range(3):
                dg = np.zeros(3)
                dg[k] = 1e-7
                J[:, k] = (resid(g + dg) - resid(g - dg)) / 2e-7
            g = g - np.linalg.solve(J, r)
        assert np.linalg.norm(resid(g)) < 1e-12 * scale
        G = pr.last["G"][0]
        P = pr.last["P"][0]
        new_states = []
        for ph, GL in enumerate(layers(g)):
            SL, st = _point_law(GL, mats[ph], states[ph])
            sel = phase == ph
            assert np.abs(G[:, :, sel] - GL[:, :, None]).max() <= 1e-7 * np.abs(GL).max(), (step, ph)
            assert np.abs(P[:, :, sel] - SL[:, :, None]).max() <= 1e-6 * np.abs(SL).max(), (step, ph)
            new_states.append(st)
        states = new_states  # committed at the end of the step, as the solver does
    # the history mattered: the second step's stress differs from a virgin response
    SA_virgin = _point_law(layers(g)[0], mats[0], _virgin_state(mats[0].law))[0]
    SA = _point_law(layers(g)[0], mats[0], states[0])[0]
    assert np.linalg.norm(P[:, :, phase == 0][:, :, 0] - SA_virgin) > 1e-3 * np.abs(SA_virgin).max()
