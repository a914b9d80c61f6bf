"""Named synthetic workloads: grid, phase map, materials, BCs, load.

A workload is plain data.  Boundary conditions are given per axis, face and
displacement component as 'P' (periodic), 'D' (Dirichlet) or 'N' (Neumann);
`bc[a][f][q]`, a = axis, f = 0 (face containing the origin) or 1, q = component.
The prescribed displacement is u*_q(x) = sum_a A[q][a] x_a + b[q] + sum_k Q[q][k] m_k(x)
with the quadratic monomials m = (x1^2, x2^2, x3^2, x2 x3, x1 x3, x1 x2) and x the
physical coordinates of the nodes (node j on axis a at j*h_a); the quadratic terms
carry bending and torsion loads.
"""

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .draws import shoemake_quaternions
from .microstructure import centred_sphere, voronoi, laminate, random_spheres

# law identifiers (same integers as the C ABI)
ISO_ELASTIC = 0
CUBIC_ELASTIC = 1
J2_LINHARD = 2
B0_LINEAR = 3  # P = 2 mu G + lambda G (.) I : the preconditioner itself (test law)
SVK_CUBIC = 4  # finite strain: St-Venant-Kirchhoff, (C11, C12, C44), quat
NEO_HOOKE = 5  # finite strain: (mu, K)
CP_FCC = 6     # finite strain crystal plasticity: (C11, C12, C44, gdot0, n, tau0, tau_inf, h0, dt), quat
LOG_J2 = 7     # finite strain perfect J2 in the logarithmic framework: (lambda, mu, sigma0)


@dataclass
class Material:
    law: int
    params: tuple  # ISO: (lambda, mu); CUBIC, SVK: (C11, C12, C44); J2: (lambda, mu, sigma_y, H); B0: (lambda, mu)
    quat: tuple = (1.0, 0.0, 0.0, 0.0)  # crystal -> sample rotation, (w, x, y, z)


@dataclass
class Workload:
    name: str
    n: tuple
    phase: np.ndarray  # uint16 [x, y, z]
    materials: List[Material]
    bc: list  # bc[axis][face][comp] in {'P','D','N'}
    scheme: str = "HEX1"  # or "TETRA2"
    green: str = "B0"  # or "MU0"
    lambda0: float = 0.0
    mu0: float = 0.0
    tol: float = 1e-8
    max_iter: int = 1000
    h: tuple = (1.0, 1.0, 1.0)
    A: np.ndarray = field(default_factory=lambda: np.zeros((3, 3)))
    b: np.ndarray = field(default_factory=lambda: np.zeros(3))
    Q: np.ndarray = field(default_factory=lambda: np.zeros((3, 6)))  # quadratic coefficients of u*_q
    anderson_depth: int = 4
    anderson_period: int = 3
    note: Optional[str] = None


def iso_lame(E, nu):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    return lam, mu


def axis_bc(x, y, z):
    """Per-axis shorthand: every face and component of an axis takes the same type."""
    return [[[t] * 3 for _ in range(2)] for t in (x, y, z)]


def sphere_inclusion_32(n=32, radius=8):
    """Two-phase sphere composite: matrix E=1, inclusion E=10, nu=0.3, HEX1, B0.

    x faces Dirichlet (all components), y Neumann, z periodic, uniaxial
    eps_xx = 1e-3 by u*_1 = eps_xx x_1; lambda0, mu0 = mean of the phases'.
    """
    nn = (n, n, n)
    phase = centred_sphere(nn, radius)
    lm = iso_lame(1.0, 0.3)
    li = iso_lame(10.0, 0.3)
    A = np.zeros((3, 3))
    A[0, 0] = 1e-3
    return Workload(
        name=f"sphere_inclusion_{n}", n=nn, phase=phase,
        materials=[Material(ISO_ELASTIC, lm), Material(ISO_ELASTIC, li)],
        bc=axis_bc("D", "N", "P"), scheme="HEX1", green="B0",
        lambda0=0.5 * (lm[0] + li[0]), mu0=0.5 * (lm[1] + li[1]),
        tol=1e-8, A=A)


def voronoi_polycrystal(n=256, grains=500, seed_geom=2, seed_orient=3,
                        scheme="TETRA2", tol=1e-6, C=(168.0, 121.0, 75.0)):
    """Cubic-elastic Voronoi polycrystal (C11=168, C12=121, C44=75 GPa).

    Grain seeds uniform in the box (seed 2), orientations uniform on SO(3)
    (seed 3).  x Dirichlet, y Neumann, z periodic, eps_xx = 1e-3.  B0 with
    lambda0 = C12 and mu0 = (C44 + (C11 - C12)/2) / 2 (mid-range shear modulus).
    """
    nn = (n, n, n) if np.isscalar(n) else tuple(n)
    phase, _ = voronoi(nn, grains, seed_geom)
    quats = shoemake_quaternions(grains, seed_orient)
    mats = [Material(CUBIC_ELASTIC, tuple(C), tuple(q)) for q in quats]
    A = np.zeros((3, 3))
    A[0, 0] = 1e-3
    C11, C12, C44 = C
    return Workload(
        name=f"voronoi_polycrystal_{nn[0]}", n=nn, phase=phase, materials=mats,
        bc=axis_bc("D", "N", "P"), scheme=scheme, green="B0",
        lambda0=C12, mu0=0.5 * (C44 + 0.5 * (C11 - C12)), tol=tol, A=A)


def x_laminate(n=(12, 4, 4), period=3, E=(1.0, 7.0), nu=(0.3, 0.2), scheme="HEX1", eps=1e-3):
    """Layers normal to x, all components Dirichlet on x, periodic y and z."""
    phase = laminate(n, 0, period)
    mats = [Material(ISO_ELASTIC, iso_lame(e, v)) for e, v in zip(E, nu)]
    lam = [m.params[0] for m in mats]
    mu = [m.params[1] for m in mats]
    A = np.zeros((3, 3))
    A[0, 0] = eps
    return Workload(
        name="x_laminate", n=tuple(n), phase=phase, materials=mats,
        bc=axis_bc("D", "P", "P"), scheme=scheme, green="B0",
        lambda0=max(lam), mu0=max(mu), tol=1e-11, A=A)


def y_laminate(n=(6, 9, 4), period=3, E=(1.0, 5.0), nu=0.25, scheme="HEX1", eps=1e-3):
    """Layers normal to y, equal Poisson ratio; normal-only Dirichlet on x
    (u_1 Dirichlet, u_2 and u_3 Neumann), traction-free y, periodic z."""
    phase = laminate(n, 1, period)
    mats = [Material(ISO_ELASTIC, iso_lame(e, nu)) for e in E]
    bc = axis_bc("D", "N", "P")
    bc[0] = [["D", "N", "N"], ["D", "N", "N"]]
    A = np.zeros((3, 3))
    A[0, 0] = eps
    lam = [m.params[0] for m in mats]
    mu = [m.params[1] for m in mats]
    return Workload(
        name="y_laminate", n=tuple(n), phase=phase, materials=mats, bc=bc,
        scheme=scheme, green="B0", lambda0=max(lam), mu0=max(mu), tol=1e-11, A=A)


def bending_load(n, h, theta):
    """Rotation theta of the x = L_1 face about the mid-line x_2 = L_2 / 2 (x = 0 at rest):
    u*_1 = (x_1 / L_1) theta (x_2 - L_2 / 2), u*_2 = u*_3 = 0.  Returns (A, b, Q)."""
    L1, L2 = n[0] * h[0], n[1] * h[1]
    A = np.zeros((3, 3))
    A[0, 0] = -theta * L2 / (2.0 * L1)
    Q = np.zeros((3, 6))
    Q[0, 5] = theta / L1  # x1 x2
    return A, np.zeros(3), Q


def rotation_e1_e3(phi, theta):
    """R = R_3(theta) R_1(phi): rotation phi about e1 (torsion) then theta about e3 (bending)."""
    c, s = np.cos(phi), np.sin(phi)
    R1 = np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])
    c, s = np.cos(theta), np.sin(theta)
    R3 = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    return R3 @ R1


def torsion_bending_load(n, h, phi, theta):
    """x = 0 at rest; the x = L_1 face turned rigidly by R = R_3(theta) R_1(phi) about its centre
    line (x2, x3) = (L2/2, L3/2), interpolated linearly in x1:
    u*(x) = (x1 / L1) (R - 1) (0, x2 - L2/2, x3 - L3/2).  Returns (A, b, Q)."""
    L1, L2, L3 = (n[a] * h[a] for a in range(3))
    W = rotation_e1_e3(phi, theta) - np.eye(3)
    A = np.zeros((3, 3))
    Q = np.zeros((3, 6))
    for q in range(3):
        Q[q, 5] = W[q, 1] / L1  # x1 x2
        Q[q, 4] = W[q, 2] / L1  # x1 x3
        A[q, 0] = -(W[q, 1] * L2 / 2.0 + W[q, 2] * L3 / 2.0) / L1
    return A, np.zeros(3), Q


def sphere_composite_bending(n=128, fraction=0.30, r_min=4.0, r_max=10.0, seed=4, scheme="HEX1",
                             E=200.0, nu=0.3, sigma_y=0.3, H=2.0, steps=20, theta_max=0.012, tol=1e-6):
    """Elasto-plastic matrix (J2, linear isotropic hardening; GPa) with elastic spherical
    particles of the same elastic moduli (overlapping random spheres, 30 % by volume, radii
    uniform in [4, 10] voxels, seed 4).  x faces Dirichlet (every component), y and z
    traction-free; bending by `bending_load` with theta_k = k theta_max / steps, k = 1..steps.
    B0 with the elastic moduli as the reference material.  Returns (workload, loads)."""
    nn = (n, n, n) if np.isscalar(n) else tuple(n)
    phase = random_spheres(nn, fraction, r_min, r_max, seed)
    lam, mu = iso_lame(E, nu)
    mats = [Material(J2_LINHARD, (lam, mu, sigma_y, H)), Material(ISO_ELASTIC, (lam, mu))]
    wl = Workload(name=f"sphere_composite_bending_{nn[0]}", n=nn, phase=phase, materials=mats,
                  bc=axis_bc("D", "N", "N"), scheme=scheme, green="B0", lambda0=lam, mu0=mu, tol=tol)
    loads = [bending_load(nn, wl.h, k * theta_max / steps) for k in range(1, steps + 1)]
    wl.A, wl.b, wl.Q = loads[0]
    return wl, loads


CP_FCC_PARAMS = (168.0, 121.0, 75.0, 1e-3, 20.0, 0.03, 0.09, 0.3, 1.0)  # C11 C12 C44 gdot0 n tau0 tau_inf h0 dt


def cp_polycrystal_torsion_bending(n=128, grains=200, seed_geom=5, seed_orient=6, increments=30, phi_final=0.05,
                                   theta_final=0.02, scheme="TETRA2", tol=1e-6):
    """Finite-strain FCC crystal plasticity (power-law slip n = 20, gdot0 = 1e-3/s, Voce hardening
    tau0 = 30 MPa, tau_inf = 90 MPa, h0 = 300 MPa; C11/C12/C44 = 168/121/75 GPa; one increment of
    1 s per load step) on a Voronoi polycrystal (grain seeds uniform in the box, seed 5; orientations
    uniform on SO(3), seed 6).  x = 0 at rest, the x = L1 face turned by the torsion-bending rotation
    R_3(theta) R_1(phi) with (phi, theta) = k (phi_final, theta_final) / increments, k = 1..increments;
    y and z traction-free; B0 with lambda0 = C12, mu0 = (C44 + (C11 - C12)/2)/2.
    Returns (workload, loads)."""
    nn = (n, n, n) if np.isscalar(n) else tuple(n)
    phase, _ = voronoi(nn, grains, seed_geom)
    quats = shoemake_quaternions(grains, seed_orient)
    mats = [Material(CP_FCC, CP_FCC_PARAMS, tuple(q)) for q in quats]
    C11, C12, C44 = CP_FCC_PARAMS[:3]
    wl = Workload(name=f"cp_polycrystal_torsion_bending_{nn[0]}", n=nn, phase=phase, materials=mats,
                  bc=axis_bc("D", "N", "N"), scheme=scheme, green="B0", lambda0=C12,
                  mu0=0.5 * (C44 + 0.5 * (C11 - C12)), tol=tol, max_iter=3000)
    loads = [torsion_bending_load(nn, wl.h, k * phi_final / increments, k * theta_final / increments)
             for k in range(1, increments + 1)]
    wl.A, wl.b, wl.Q = loads[0]
    return wl, loads

