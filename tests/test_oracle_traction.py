"""Non-zero Neumann tractions in the oracle (Sec. 2.2: P = P^f + P*, P* = 2 t at the mirror
voxel centres of a loaded face), pinned by closed forms.

* The imposed stress alone: for P^f = 0 both stencils give D* = 2 t_q / h_a at the nodes of
  a loaded face away from its edges (the two ghost corners of each divergence pair, weight
  1/(4 h) x 4 pairs for HEX1, 1/(2 h) x 2 pairs averaged over the two TETRA2 pairings), zero
  in the interior, nothing on a Dirichlet component.
* An end-loaded homogeneous bar (x = 0 face: u_1 = 0, everything else traction-free except
  t_1 = sigma on x = L) has the affine uniaxial-stress solution, which both stencils
  reproduce exactly: eps_11 = sigma / E, eps_22 = eps_33 = -nu sigma / E, P = sigma e1 (x) e1.
"""

import numpy as np
import pytest

import synthetic as syn
from oracle.bc import Grid
from oracle.solver import Problem
from oracle.stencils import div
from synthetic.workloads import ISO_ELASTIC, Material, Workload


def _bar_bc():
    # x: comp 1 Dirichlet on the x = 0 face only; all else Neumann
    return [[["D", "N", "N"], ["N", "N", "N"]], [["N"] * 3, ["N"] * 3], [["N"] * 3, ["N"] * 3]]


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_imposed_stress_gives_two_t_over_h_on_a_loaded_face(scheme):
    n, h = (6, 5, 4), (1.0, 0.5, 2.0)
    g = Grid(n, _bar_bc(), h)
    npp = 1 if scheme == "HEX1" else 2
    T = np.zeros((3, 2, 3))
    T[0, 1] = (0.7, -0.3, 0.2)  # x = L face, all three components Neumann there
    T[0, 0] = (0.5, 0.0, 0.0)  # x = 0 face: component 1 is Dirichlet, must be ignored
    D = div(np.zeros((npp, 3, 3) + n), g, scheme, T)
    N = g.N
    inner = (slice(1, N[1] - 1), slice(1, N[2] - 1))
    for q in range(3):
        assert np.allclose(D[q][N[0] - 1][inner], 2.0 * T[0, 1, q] / h[0], rtol=1e-14, atol=0)
        assert np.abs(D[q][1:N[0] - 1]).max() == 0.0
    assert np.abs(D[0][0]).max() == 0.0


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_end_loaded_bar_is_in_uniaxial_stress(scheme):
    E, nu, sig = 2.0, 0.3, 1e-3
    lam, mu = syn.iso_lame(E, nu)
    n = (8, 6, 6)
    T = np.zeros((3, 2, 3))
    T[0, 1, 0] = sig
    wl = Workload("bar_traction", n, np.zeros(n, np.uint16), [Material(ISO_ELASTIC, (lam, mu))], _bar_bc(),
                  scheme=scheme, lambda0=lam, mu0=mu, tol=1e-12, A=np.zeros((3, 3)), max_iter=3000)
    pr = Problem(wl)
    uf, rep = pr.solve_step(T=T)
    assert rep.converged
    G = pr.last["G"]
    eps = 0.5 * (G + np.swapaxes(G, 1, 2))
    expect = np.diag([sig / E, -nu * sig / E, -nu * sig / E])
    assert np.abs(eps - expect[None, :, :, None, None, None]).max() < 1e-10 * sig / E
    P = pr.last["P"]
    assert np.abs(P - np.diag([sig, 0.0, 0.0])[None, :, :, None, None, None]).max() < 1e-10 * sig
