"""Finite-strain oracle laws pinned by closed forms (Sec. 3.1.2, Sec. 3.4, Appendix B).

* St-Venant-Kirchhoff, cubic axes aligned: a bar under uniaxial stress has the
  closed form worked out below (lateral Green-Lagrange strain from Pi_22 = 0).
* Neo-Hookean: the uniaxial closed form of Appendix B (P11 and P22 in terms of the
  longitudinal and transverse stretches), transverse stretch from P22 = 0 (with the
  bulk term of P22 re-derived, see the comment in the test).
  Both are solved through the fixed point (homogeneous bar, normal-only Dirichlet on
  x, traction-free elsewhere), so they also pin F = 1 + grad u and P = F Pi.
* Crystal plasticity: one slip system (m = e1, n = e2) under simple shear
  F = 1 + gamma e1 (x) e2 with aligned cubic elasticity reduces exactly to a scalar
  recursion for the slip, tau = C44 (gamma - gamma_p); it is solved here by bracketing.
"""

import numpy as np
import pytest
from scipy.optimize import brentq

import synthetic as syn
from oracle import finite
from oracle.solver import Problem
from synthetic.workloads import Material, Workload, axis_bc


def _bar(law, params, scheme, quat=(1.0, 0.0, 0.0, 0.0), lam0=121.0, mu0=75.0):
    n = (6, 4, 4)
    bc = axis_bc("D", "N", "N")
    bc[0] = [["D", "N", "N"], ["D", "N", "N"]]
    return Workload("bar", n, np.zeros(n, np.uint16), [Material(law, params, quat)], bc, scheme=scheme,
                    lambda0=lam0, mu0=mu0, tol=1e-12, max_iter=3000)


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_svk_bar_uniaxial_closed_form(scheme):
    C11, C12, C44 = 168.0, 121.0, 75.0
    wl = _bar(syn.workloads.SVK_CUBIC, (C11, C12, C44), scheme)
    pr = Problem(wl)
    for e in (1.02, 1.05):
        A = np.zeros((3, 3))
        A[0, 0] = e - 1.0
        _, rep = pr.solve_step(A=A)
        assert rep.converged, rep.err[-3:]
        E1 = 0.5 * (e * e - 1.0)
        E2 = -C12 * E1 / (C11 + C12)  # Pi_22 = C12 E1 + (C11 + C12) E2 = 0
        P11 = e * (C11 * E1 + 2.0 * C12 * E2)
        S = pr.last["P"]  # S[i, q] = P_qi
        assert np.abs(S[:, 0, 0] - P11).max() < 1e-9 * P11
        assert np.abs(S[:, 1, 1]).max() < 1e-9 * P11 and np.abs(S[:, 2, 2]).max() < 1e-9 * P11
        eT = np.sqrt(1.0 + 2.0 * E2)
        G = pr.last["G"]
        assert np.allclose(G[:, 1, 1], eT - 1.0, rtol=0, atol=1e-10)


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_neo_hooke_bar_matches_the_appendix_b_closed_form(scheme):
    mu, K = 0.6, 1.5
    # reference material 1.5x the small-strain moduli (the finite-strain tangent stiffens in tension)
    wl = _bar(syn.workloads.NEO_HOOKE, (mu, K), scheme, lam0=1.5 * (K - 2 * mu / 3), mu0=1.5 * mu)

    def p11(e, eT):
        return 2.0 / 3.0 * mu * eT ** 2 * (e * eT ** 2) ** (-5.0 / 3.0) * (e ** 2 - eT ** 2) + K * (e * eT ** 4 - eT ** 2)

    # Appendix B prints the bulk term of P22 as K e eT (eT^2 - 1); the same energy gives
    # P22 = e eT sigma_22 with sigma_22 = mu J^(-5/3) (eT^2 - e^2) / 3 + K (J - 1), J = e eT^2,
    # i.e. K e eT (e eT^2 - 1), which is also the only form consistent with the printed P11
    def p22(e, eT):
        return 1.0 / 3.0 * mu * e * eT * (e * eT ** 2) ** (-5.0 / 3.0) * (eT ** 2 - e ** 2) + K * e * eT * (e * eT ** 2 - 1.0)

    pr = Problem(wl)
    for e in (1.05, 1.2):
        A = np.zeros((3, 3))
        A[0, 0] = e - 1.0
        _, rep = pr.solve_step(A=A)
        assert rep.converged, rep.err[-3:]
        eT = brentq(lambda t: p22(e, t), 0.5, 1.0)
        S = pr.last["P"]
        assert np.abs(S[:, 0, 0] - p11(e, eT)).max() < 1e-8 * p11(e, eT)
        assert np.abs(S[:, 1, 1]).max() < 1e-8 * p11(e, eT)
        assert np.allclose(pr.last["G"][:, 1, 1], eT - 1.0, rtol=0, atol=1e-9)


def test_fcc_slip_systems_are_the_twelve_111_110_systems():
    m, n = finite.fcc_slip_systems()
    assert m.shape == (12, 3) and n.shape == (12, 3)
    assert np.allclose(np.abs(m @ n.T).diagonal(), 0.0)
    assert np.allclose(np.linalg.norm(m, axis=1), 1.0) and np.allclose(np.linalg.norm(n, axis=1), 1.0)
    assert np.allclose(np.sort(np.abs(n * np.sqrt(3)), axis=1), 1.0)  # {111}
    assert np.allclose(np.sort(np.abs(m * np.sqrt(2)), axis=1), [0.0, 1.0, 1.0])  # <110>
    pairs = {(tuple(np.round(a, 9)), tuple(np.round(b, 9))) for a, b in zip(m, n)}
    assert len(pairs) == 12


def test_single_slip_simple_shear_follows_the_scalar_recursion():
    C11, C12, C44 = 168.0, 121.0, 75.0
    gdot0, nexp, tau0, tau_inf, h0, dt = 1e-3, 20.0, 0.03, 0.09, 0.3, 1.0
    C = finite.rotated_cubic((C11, C12, C44), (1.0, 0.0, 0.0, 0.0))
    Ps = np.zeros((1, 3, 3))
    Ps[0, 0, 1] = 1.0  # m = e1, n = e2
    Fp = np.eye(3)[None].copy()
    gam = np.zeros(1)
    gp = 0.0  # scalar recursion state
    for k in range(1, 16):
        g = 2e-4 * k
        F = np.eye(3)[None].copy()
        F[0, 0, 1] = g
        P, Fp, gam_new, it = finite.cp_update(F, Fp, gam, C, Ps, gdot0, nexp, tau0, tau_inf, h0, dt)
        tauc = tau0 + (tau_inf - tau0) * (1.0 - np.exp(-h0 * gp / (tau_inf - tau0)))
        g_tr = g - gp
        f = lambda d: d - dt * gdot0 * (max(C44 * (g_tr - d), 0.0) / tauc) ** nexp
        d = brentq(f, 0.0, max(g_tr, 1e-30)) if g_tr > 0 else 0.0
        gp += d
        assert abs(Fp[0, 0, 1] - gp) < 1e-10 + 1e-8 * gp, (k, Fp[0, 0, 1], gp)
        assert abs(gam_new[0] - gp) < 1e-10 + 1e-8 * gp
        Fe = F[0] @ np.linalg.inv(Fp[0])
        Pi = np.linalg.solve(Fe, P[0]) @ Fp[0].T  # P = F^e Pi F^p^-T
        assert abs(Pi[0, 1] - C44 * (g - gp)) < 1e-9 * C44 * g
        gam = gam_new
    assert gp > 1e-3  # the recursion went well into the plastic range
