"""Named synthetic workloads: grid, phase map, materials, BCs, load.

A workload is plain data.  Boundary conditions are given per axis, face and
displacement component as 'P' (periodic), 'D' (Dirichlet) or 'N' (Neumann);
`bc[a][f][q]`, a = axis, f = 0 (face containing the origin) or 1, q = component.
The prescribed displacement is u*_q(x) = sum_a A[q][a] x_a + b[q] + B[q] x_1 x_2,
with x the physical coordinates of the nodes (node j on axis a at j*h_a); the
bilinear term carries the bending loads.
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


@dataclass
class Material:
    law: int
    params: tuple  # ISO: (lambda, mu); CUBIC: (C11, C12, C44); J2: (lambda, mu, sigma_y, H); B0: (lambda, mu)
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
    B: np.ndarray = field(default_factory=lambda: np.zeros(3))  # coefficient of x_1 x_2 in u*_q
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
    u*_1 = (x_1 / L_1) theta (x_2 - L_2 / 2), u*_2 = u*_3 = 0.  Returns (A, b, B)."""
    L1, L2 = n[0] * h[0], n[1] * h[1]
    A = np.zeros((3, 3))
    A[0, 0] = -theta * L2 / (2.0 * L1)
    B = np.zeros(3)
    B[0] = theta / L1
    return A, np.zeros(3), B


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
    wl.A, wl.b, wl.B = loads[0]
    return wl, loads
