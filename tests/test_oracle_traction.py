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
from synthetic.workloads import ISO_ELASTIC, Material, Workload, axis_bc


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


def test_face_field_gives_the_hand_derived_nodal_forces():
    """Non-uniform tractions t(v_b, v_c) on one face: with the stress itself zero, the HEX1
    divergence at a node (m_b, m_c) of the face is the average over its four face voxels of
    2 t / h_a (the uniform case's 2 t / h_a, voxel by voxel), the voxels beyond the face's
    edges taking the value of the face voxel they mirror; the other faces' nodes get nothing."""
    n = (6, 5, 4)
    h = (1.0, 0.8, 1.3)
    bc = axis_bc("D", "N", "N")
    g = Grid(n, bc, h)
    rng = np.random.default_rng(3)
    t = rng.standard_normal((3, n[0], n[2]))  # face y = L2 (axis 1, face 1): in-plane axes x, z
    D = div(np.zeros((1, 3, 3) + n), g, "HEX1", Tf={(1, 1): t})
    for q in range(3):
        for mb in range(n[0] + 1):
            for mc in range(n[2] + 1):
                vals = [t[q, min(max(mb + ob - 1, 0), n[0] - 1), min(max(mc + oc - 1, 0), n[2] - 1)]
                        for ob in (0, 1) for oc in (0, 1)]
                assert abs(D[q, mb, n[1], mc] - 2.0 / h[1] * np.mean(vals)) < 1e-12
    assert np.abs(D[:, :, : n[1], :]).max() < 1e-12


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_uniform_face_field_equals_the_uniform_traction(scheme):
    n = (6, 5, 4)
    g = Grid(n, axis_bc("D", "N", "N"), (1.0, 0.8, 1.3))
    S = np.random.default_rng(4).standard_normal((2 if scheme == "TETRA2" else 1, 3, 3) + n)
    T = np.zeros((3, 2, 3))
    T[2, 0] = [0.3, -0.2, 0.5]
    field = np.broadcast_to(np.array(T[2, 0])[:, None, None], (3, n[0], n[1])).copy()
    a = div(S, g, scheme, T=T)
    b = div(S, g, scheme, Tf={(2, 0): field})
    assert np.abs(a - b).max() < 1e-12
