"""Normal-mixed loading (Eq. NMBC1) in the oracle, pinned by closed forms and by an exact
superposition of direct sparse solves.

* The increment of the free strain components is exact in one step when the reference
  material is the material itself (a homogeneous medium): the isotropic uniaxial-stress
  state.
* A homogeneous isotropic medium under NMBC1 with only eps_11 imposed converges to the
  uniaxial-stress closed form (eps_22 = eps_33 = -nu eps_11, sigma_11 = E eps_11).
* A two-phase linear medium: the mixed problem is linear in the free strain components,
  so its exact solution is the imposed-strain solution plus the combination of unit-strain
  solutions (each a direct sparse solve of the discrete system) that cancels the free
  mean stresses; the iterative mixed solve must reproduce its strain of u* and its strain
  field (the displacement only up to the stencils' zero-gradient modes).
"""

import numpy as np
import pytest

import synthetic as syn
from oracle import direct
from oracle.mixed import VOIGT, free_components, mixed_error, mixed_increment, nmbc1_bc
from oracle.solver import Problem
from synthetic.workloads import ISO_ELASTIC, Material, Workload

ALL_BUT_11 = 0b111110


def _iso_sigma(eps, lam, mu):
    return lam * np.trace(eps) * np.eye(3) + 2.0 * mu * eps


def test_increment_is_exact_with_the_material_as_reference():
    lam, mu = syn.iso_lame(1.0, 0.3)
    eps0 = np.zeros((3, 3))
    eps0[0, 0] = 1e-3
    eps0[0, 1] = eps0[1, 0] = 2e-4  # a shear the mask frees as well
    d = mixed_increment(_iso_sigma(eps0, lam, mu), ALL_BUT_11, lam, mu)
    s = _iso_sigma(eps0 + d, lam, mu)
    for k in free_components(ALL_BUT_11):
        i, j = VOIGT[k]
        assert abs(s[i, j]) < 1e-15
    assert abs(d[0, 0]) == 0.0
    assert np.isclose((eps0 + d)[1, 1], -0.3 * 1e-3, rtol=1e-12)
    assert np.isclose(s[0, 0], 1e-3, rtol=1e-12)  # E eps with E = 1
    assert mixed_error(s, ALL_BUT_11) < 1e-12 and mixed_error(_iso_sigma(eps0, lam, mu), ALL_BUT_11) > 0.1


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_nmbc1_homogeneous_medium_is_in_uniaxial_stress(scheme):
    E, nu, eps = 1.0, 0.3, 1e-3
    lam, mu = syn.iso_lame(E, nu)
    n = (6, 5, 4)
    A = np.zeros((3, 3))
    A[0, 0] = eps
    # a reference material away from the medium, so that the adjustment takes iterations
    wl = Workload("nmbc1_homog", n, np.zeros(n, np.uint16), [Material(ISO_ELASTIC, (lam, mu))], nmbc1_bc(),
                  scheme=scheme, lambda0=1.4 * lam, mu0=1.3 * mu, tol=1e-12, A=A, max_iter=3000)
    pr = Problem(wl)
    uf, rep = pr.solve_step(mixed=ALL_BUT_11)
    assert rep.converged and rep.iterations > 2
    expect = np.diag([eps, -nu * eps, -nu * eps])
    assert np.abs(rep.A - expect).max() < 1e-11
    assert np.abs(rep.mean_P - np.diag([E * eps, 0.0, 0.0])).max() < 1e-11
    assert np.abs(uf).max() < 1e-11


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_nmbc1_two_phase_matches_superposed_direct_solves(scheme):
    n = (8, 6, 6)
    lam1, mu1 = syn.iso_lame(1.0, 0.3)
    lam2, mu2 = syn.iso_lame(8.0, 0.25)
    ph = syn.centred_sphere(n, 2)
    mats = [Material(ISO_ELASTIC, (lam1, mu1)), Material(ISO_ELASTIC, (lam2, mu2))]
    eps = 1e-3

    def workload(A):
        return Workload("nmbc1_2ph", n, ph, mats, nmbc1_bc(), scheme=scheme, lambda0=0.5 * (lam1 + lam2),
                        mu0=0.5 * (mu1 + mu2), tol=1e-11, A=A, max_iter=5000)

    # unit symmetric strains of u* and their direct solutions
    units, sols, sig = [], [], []
    for k in range(6):
        Ek = np.zeros((3, 3))
        i, j = VOIGT[k]
        Ek[i, j] = Ek[j, i] = 1.0
        wk = workload(Ek)
        pk = Problem(wk)
        Gs = pk.grad_ustar()
        uk = direct.solve(wk, Gs)
        P = pk.residual(uk, Gs)[2]
        Pm = P.mean(axis=(0, 3, 4, 5))
        units.append(Ek)
        sols.append(uk)
        sig.append(0.5 * (Pm + Pm.T))
    F = free_components(ALL_BUT_11)
    M = np.array([[sig[k][VOIGT[f]] for k in F] for f in F])
    rhs = np.array([-eps * sig[0][VOIGT[f]] for f in F])
    x = np.linalg.solve(M, rhs)
    A_exact = eps * units[0] + sum(xk * units[k] for xk, k in zip(x, F))
    u_exact = eps * sols[0] + sum(xk * sols[k] for xk, k in zip(x, F))

    A0 = np.zeros((3, 3))
    A0[0, 0] = eps
    pr = Problem(workload(A0))
    uf, rep = pr.solve_step(mixed=ALL_BUT_11)
    assert rep.converged
    assert np.abs(rep.A - A_exact).max() < 1e-8 * eps
    # strains, not displacements: under NMBC1 the stencils keep zero-gradient (hourglass)
    # modes, which the direct solve and the fixed point (null rule) settle differently
    e1 = pr.residual(uf, pr.grad_ustar(rep.A))[3]
    e2 = pr.residual(u_exact, pr.grad_ustar(A_exact))[3]
    e1, e2 = e1 + np.swapaxes(e1, 1, 2), e2 + np.swapaxes(e2, 1, 2)
    assert np.abs(e1 - e2).max() < 1e-8 * np.abs(e2).max()
    assert rep.mixed_err[-1] < 1e-11
