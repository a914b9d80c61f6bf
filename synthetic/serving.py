"""The serving request stream: independent solves of mixed sizes, boundary conditions,
laws and schemes (seeded; no solver arithmetic).

Request k uses the seed 1000 + k and draws, uniformly and independently:
* grid side n in {32, 48, 64, 96, 128} (n^3 voxels);
* a boundary condition per axis in {P, D, N}; draws without a Dirichlet axis are
  redrawn (the load is an imposed displacement on a Dirichlet axis; periodic axes
  cannot carry one);
* the matrix law: isotropic elastic (E = 200 GPa, nu = 0.3) or J2 with linear
  hardening (same elasticity, sigma_y = 0.3 GPa, H = 2 GPa);
* the scheme: HEX1 or TETRA2;
* the microstructure: random spheres (30 % by volume, radii in [n/32, n/12.8]
  voxels, i.e. [4, 10] at 128^3) or a Voronoi tessellation of n/4 grains with the
  grains split between the two phases by grain index parity; the second phase is
  elastic with E = 400 GPa, nu = 0.3.
Loading: normal strain 1e-3 on the first Dirichlet axis a (u*_a = 1e-3 x_a), one load
step for elastic matrices, two (1e-3 then 2e-3, past the matrix's yield strain of
1.5e-3) for J2.  Reference material: half the sum of the phases' largest and
smallest Lame constants.  Tolerance 1e-6.
"""

import numpy as np

from .microstructure import random_spheres, voronoi
from .workloads import ISO_ELASTIC, J2_LINHARD, Material, Workload, iso_lame

SIDES = (32, 48, 64, 96, 128)


def request_spec(k):
    rng = np.random.default_rng(1000 + k)
    side = int(rng.choice(SIDES))
    while True:
        bcs = [str(rng.choice(["P", "D", "N"])) for _ in range(3)]
        if "D" in bcs:
            break
    return {
        "index": k,
        "seed": 1000 + k,
        "n": side,
        "bc": bcs,
        "law": "J2" if rng.random() < 0.5 else "ISO",
        "scheme": "TETRA2" if rng.random() < 0.5 else "HEX1",
        "micro": "voronoi" if rng.random() < 0.5 else "spheres",
    }


def request_workload(spec):
    """Workload and load list of one request."""
    n = spec["n"]
    nn = (n, n, n)
    if spec["micro"] == "spheres":
        phase = random_spheres(nn, 0.30, n / 32.0, n / 12.8, spec["seed"])
    else:
        grains, _ = voronoi(nn, max(4, n // 4), spec["seed"])
        phase = (grains % 2).astype(np.uint16)
    lam, mu = iso_lame(200.0, 0.3)
    lam2, mu2 = iso_lame(400.0, 0.3)
    matrix = Material(J2_LINHARD, (lam, mu, 0.3, 2.0)) if spec["law"] == "J2" else Material(ISO_ELASTIC, (lam, mu))
    mats = [matrix, Material(ISO_ELASTIC, (lam2, mu2))]
    bc = [[[t] * 3 for _ in range(2)] for t in spec["bc"]]
    a = spec["bc"].index("D")
    strains = (1e-3, 2e-3) if spec["law"] == "J2" else (1e-3,)
    loads = []
    for eps in strains:
        A = np.zeros((3, 3))
        A[a, a] = eps
        loads.append((A, np.zeros(3), np.zeros((3, 6))))
    wl = Workload(name=f"request_{spec['index']}", n=nn, phase=phase, materials=mats, bc=bc,
                  scheme=spec["scheme"], green="B0", lambda0=0.5 * (lam + lam2), mu0=0.5 * (mu + mu2),
                  tol=1e-6, max_iter=2000, A=loads[0][0])
    return wl, loads
