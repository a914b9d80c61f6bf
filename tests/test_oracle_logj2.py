"""The logarithmic finite-strain J2 law of the oracle (Sec. 3.2, the porous-medium law),
pinned without the law's own machinery.

* Pure stretch F = diag(a, b, c) below yield: H = diag(log a, log b, log c), and the
  first Piola stress is diagonal with P_aa = T_aa / a (S_aa = T_aa / a^2), T = 2 mu dev H +
  K tr H 1.
* Below yield S is the derivative of the stored energy psi = mu dev H : dev H +
  K/2 (tr H)^2 with respect to E = (C - 1)/2: central differences of psi computed with
  scipy's matrix logarithm (not the law's eigenbasis formula).
* Objectivity: P(Q F) = Q P(F) for a rotation Q, elastic and plastic.
* After a plastic step the return lands on the yield surface (T_eq = sigma0) and the
  plastic Hencky strain is deviatoric; at small strain the law tends to small-strain
  perfect J2 (the J2 law with H = 0).
"""

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import finite
from oracle.laws import j2_return

LAM, MU, SIG0 = 1.2, 0.8, 2e-3
K = LAM + 2 * MU / 3
PARAMS = (LAM, MU, SIG0)


def _G_of_F(F):
    """F (3, 3) -> G (1, 3, 3, 1) with G[i, q] = F[q, i] - delta."""
    return (F - np.eye(3)).T[None, :, :, None]


def _P_of(F, Hp=None, p=None):
    S, Hp1, p1 = finite.log_j2(_G_of_F(F), PARAMS, np.zeros((1, 3, 3, 1)) if Hp is None else Hp,
                               np.zeros((1, 1)) if p is None else p)
    return S[0, :, :, 0].T, Hp1, p1  # P[q, i]


def _rotation(seed):
    q = np.random.default_rng(seed).standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_pure_stretch_below_yield_closed_form():
    st = np.array([1.0004, 0.9998, 1.0001])
    P, _, p = _P_of(np.diag(st))
    H = np.log(st)
    T = 2 * MU * (H - H.mean()) + K * H.sum()
    assert np.allclose(np.diag(P), T / st, rtol=1e-9, atol=0)  # T_22 is a small difference: ~1e-11 rounding
    assert np.abs(P - np.diag(np.diag(P))).max() < 1e-18 and p[0, 0] == 0.0


def test_stress_is_the_energy_derivative_below_yield():
    rng = np.random.default_rng(3)
    F = np.eye(3) + 3e-4 * rng.standard_normal((3, 3))

    def psi(E):
        Hm = 0.5 * sla.logm(2.0 * E + np.eye(3)).real
        tr = np.trace(Hm)
        d = Hm - tr / 3 * np.eye(3)
        return MU * np.sum(d * d) + 0.5 * K * tr * tr

    E0 = 0.5 * (F.T @ F - np.eye(3))
    S_fd = np.zeros((3, 3))
    h = 1e-7
    for i in range(3):
        for j in range(i, 3):
            dE = np.zeros((3, 3))
            dE[i, j] = dE[j, i] = h if i != j else h
            d = (psi(E0 + dE) - psi(E0 - dE)) / (2 * h)
            S_fd[i, j] = S_fd[j, i] = d if i == j else d / 2  # d psi / d E_ij counts both entries
    P, _, _ = _P_of(F)
    S = np.linalg.solve(F, P)
    assert np.abs(S - S_fd).max() < 1e-6 * np.abs(S_fd).max()


@pytest.mark.parametrize("amp", [3e-4, 2e-2])  # elastic, plastic
def test_objectivity(amp):
    rng = np.random.default_rng(11)
    F = np.eye(3) + amp * rng.standard_normal((3, 3))
    Q = _rotation(4)
    P1, Hp1, p1 = _P_of(F)
    P2, Hp2, p2 = _P_of(Q @ F)
    assert np.abs(P2 - Q @ P1).max() < 1e-12 * np.abs(P1).max()
    assert np.abs(Hp2 - Hp1).max() < 1e-12 and abs(p2[0, 0] - p1[0, 0]) < 1e-14


def test_plastic_return_is_on_the_yield_surface_and_deviatoric():
    rng = np.random.default_rng(12)
    F = np.eye(3) + 2e-2 * rng.standard_normal((3, 3))
    P, Hp, p = _P_of(F)
    assert p[0, 0] > 0
    C = F.T @ F
    H = 0.5 * sla.logm(C).real
    He = H - Hp[0, :, :, 0]
    T = 2 * MU * (He - np.trace(He) / 3 * np.eye(3)) + K * np.trace(He) * np.eye(3)
    s = T - np.trace(T) / 3 * np.eye(3)
    assert abs(np.sqrt(1.5 * np.sum(s * s)) - SIG0) < 1e-12
    assert abs(np.trace(Hp[0, :, :, 0])) < 1e-15


def test_small_strain_limit_is_perfect_j2():
    rng = np.random.default_rng(13)
    A = rng.standard_normal((3, 3))
    for eps in (1e-5, 1e-6):
        F = np.eye(3) + eps * 400 * A  # well past yield at both sizes (sigma0 / (2 mu) = 1.25e-3)
        P, _, _ = _P_of(F)
        e = 0.5 * ((F - np.eye(3)) + (F - np.eye(3)).T)
        sig, _, _ = j2_return(e[None, :, :, None], np.zeros((1, 3, 3, 1)), np.zeros((1, 1)), LAM, MU, SIG0, 0.0)
        sig = sig[0, :, :, 0]
        # first order in the strain (4e-4 A and 4e-3 A): the gap shrinks with the strain
        rel = np.abs(P - sig).max() / np.abs(sig).max()
        assert rel < 40 * eps * 400 * np.abs(A).max(), (eps, rel)


@pytest.mark.parametrize("a", [1.0005, 1.004])  # elastic, past yield
def test_homogeneous_bar_through_the_fixed_point(a):
    """x faces: u_1 imposed (stretch a), tangential components free; y and z faces free.
    The homogeneous bar is in uniaxial Hencky stress: elastic, H_22 = H_33 = -nu log a;
    past yield, T = diag(sigma0, 0, 0), H^e_11 = sigma0 / E, H^p deviatoric, so
    H_22 = -nu sigma0 / E - (log a - sigma0 / E) / 2.  P = diag(T_11 / a, 0, 0)."""
    from oracle.solver import Problem
    from synthetic.workloads import LOG_J2, Material, Workload

    n = (6, 4, 4)
    bc = [[["D", "N", "N"], ["D", "N", "N"]], [["N"] * 3, ["N"] * 3], [["N"] * 3, ["N"] * 3]]
    A = np.zeros((3, 3))
    A[0, 0] = a - 1.0
    wl = Workload("logj2_bar", n, np.zeros(n, np.uint16), [Material(LOG_J2, PARAMS)], bc, scheme="HEX1",
                  lambda0=LAM, mu0=MU, tol=1e-11, A=A, max_iter=4000)
    pr = Problem(wl)
    _, rep = pr.solve_step()
    assert rep.converged
    E = MU * (3 * LAM + 2 * MU) / (LAM + MU)
    nu = LAM / (2 * (LAM + MU))
    la = np.log(a)
    if E * la <= SIG0:
        h22, t11 = -nu * la, E * la
    else:
        h22, t11 = -nu * SIG0 / E - 0.5 * (la - SIG0 / E), SIG0
    b = np.exp(h22)
    G = pr.last["G"]
    Fexp = np.diag([a, b, b])
    Gexp = (Fexp - np.eye(3)).T
    assert np.abs(G - Gexp[None, :, :, None, None, None]).max() < 1e-9
    P = pr.last["P"]  # S[i, q] = P[q, i]; diagonal here
    Pexp = np.diag([t11 / a, 0.0, 0.0])
    assert np.abs(P - Pexp[None, :, :, None, None, None]).max() < 1e-9 * SIG0
