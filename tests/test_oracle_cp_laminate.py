"""Pin of the oracle's full-field crystal-plasticity solve against an independent construction.

A laminate of two FCC crystals (layers normal to x, three voxels each, Dirichlet x faces,
periodic y and z) under an affine displacement u* = A x that depends on x only has a
displacement fluctuation depending on x only, piecewise linear with kinks at the interfaces:
the HEX1 gradient is then exact in every voxel, the gradient of each layer is
G_L = G* + e1 (x) g_L with the zero-mean condition n_A g_A + n_B g_B = 0 (u^f vanishes on both
x faces), and the divergence vanishes everywhere iff the traction on the interface planes is
continuous, S_A[0, :] = S_B[0, :] (Eq. GeneralBCtobesolved with the stencils of Sec. 2.5).  The
test solves those three equations for g_A by its own Newton iteration, with the oracle's
pointwise law (`oracle.finite.cp_fcc`, pinned separately by the single-slip recursion) from the
virgin state, and compares with Algorithm 1 run by the oracle on the full grid: one implicit
increment past yield (power-law slip with Voce hardening, the crystal law of Sec. 3.4 as the
oracle states it)."""

import numpy as np

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
