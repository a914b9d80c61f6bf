"""Finite-strain laws and quadratic loads on the GPU against the oracle (through the C ABI).

* quadratic u*: the total gradient the library evaluates for every monomial of
  u* (both schemes) equals the oracle's stencil applied to u* on the node grid;
* St-Venant-Kirchhoff and Neo-Hookean bars in uniaxial tension: the fixed point
  reproduces the closed forms (the same problems pin the oracle);
* a cubic St-Venant-Kirchhoff polycrystal under torsion-bending (quadratic u*),
  two load steps: FP64 with the oracle's iteration counts and fields to 1e-9,
  FP32 within one Anderson period (+-3 iterations) and 1e-5 relative L2.
"""

import numpy as np
import pytest

import synthetic as syn
from abi_helpers import GpuProblem, rel_l2
from oracle.solver import Problem
from paper_2607_05929_gb300 import build
from paper_2607_05929_gb300 import fftm as F
from synthetic.workloads import ISO_ELASTIC, NEO_HOOKE, SVK_CUBIC, Material, Workload, axis_bc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    F.load_library()


def _s9(S):
    """oracle S (npp, 3, 3, n1, n2, n3) -> (npp, 9, ...) with c = 3 i + q."""
    return S.reshape(S.shape[0], 9, *S.shape[3:])


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_quadratic_load_gradient_matches_the_oracle(scheme):
    n = (8, 6, 4)
    rng = np.random.default_rng(5)
    A = 1e-3 * rng.standard_normal((3, 3))
    Q = 1e-4 * rng.standard_normal((3, 6))
    wl = Workload("quad", n, np.zeros(n, np.uint16), [Material(ISO_ELASTIC, (1.0, 1.0))], axis_bc("D", "N", "N"),
                  scheme=scheme, lambda0=1.0, mu0=1.0, A=A, Q=Q, h=(1.0, 0.8, 1.3))
    pr = Problem(wl)
    gp = GpuProblem(wl, "fp64")
    try:
        Gg = gp.get_voxel(F.FFTM_FIELD_GRAD)  # u^f = 0: the gradient of u* alone
        Go = pr.grad_ustar()
        assert rel_l2(Gg, Go.reshape(Go.shape[0], 9, *Go.shape[3:])) < 1e-13
    finally:
        gp.close()


def _bar(law, params, scheme, lam0, mu0):
    n = (6, 4, 4)
    bc = axis_bc("D", "N", "N")
    bc[0] = [["D", "N", "N"], ["D", "N", "N"]]
    return Workload("bar", n, np.zeros(n, np.uint16), [Material(law, params)], bc, scheme=scheme,
                    lambda0=lam0, mu0=mu0, tol=1e-11, max_iter=3000)


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_svk_and_neo_hooke_bars_match_the_oracle(scheme):
    cases = [(SVK_CUBIC, (168.0, 121.0, 75.0), 121.0, 75.0, (1.02, 1.05)),
             (NEO_HOOKE, (0.6, 1.5), 1.5 * (1.5 - 0.4), 0.9, (1.05, 1.2))]
    for law, params, lam0, mu0, stretches in cases:
        wl = _bar(law, params, scheme, lam0, mu0)
        pr = Problem(wl)
        gp = GpuProblem(wl, "fp64")
        try:
            for e in stretches:
                A = np.zeros((3, 3))
                A[0, 0] = e - 1.0
                _, rep = pr.solve_step(A=A)
                gp.set_load(A, np.zeros(3), None)
                st, r, eh, ah = F.fftm_solve_step(gp.p, history_len=wl.max_iter + 1)
                assert st == F.FFTM_OK and r["converged"]
                assert abs(r["iterations"] - rep.iterations) <= 2, (law, e, r["iterations"], rep.iterations)
                Sg = gp.get_voxel(F.FFTM_FIELD_STRESS)
                assert rel_l2(Sg, _s9(pr.last["P"])) < 1e-9, (law, e)
        finally:
            gp.close()


def _poly(scheme, tol):
    n = (16, 12, 8)
    ph, _ = syn.voronoi(n, 6, 7)
    quats = syn.shoemake_quaternions(6, 8)
    mats = [Material(SVK_CUBIC, (168.0, 121.0, 75.0), tuple(q)) for q in quats]
    loads = [syn.torsion_bending_load(n, (1.0, 1.0, 1.0), k * 0.05 / 2, k * 0.02 / 2) for k in (1, 2)]
    wl = Workload("svk_tb", n, ph, mats, axis_bc("D", "N", "N"), scheme=scheme, lambda0=121.0, mu0=75.0,
                  tol=tol, max_iter=2000)
    return wl, loads


# TETRA2 only: with HEX1 this finite-strain torsion-bending problem does not converge (in the
# oracle as in the library), the behaviour the paper reports for HEX1 under finite strain
@pytest.mark.parametrize("scheme", ["TETRA2"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_svk_polycrystal_torsion_bending_matches_the_oracle(scheme, precision):
    wl, loads = _poly(scheme, 1e-8 if precision == "fp64" else 1e-6)
    pr = Problem(wl)
    gp = GpuProblem(wl, precision)
    try:
        for k, (A, b, Q) in enumerate(loads):
            _, rep = pr.solve_step(A=A, b=b, Q=Q)
            assert rep.converged
            gp.set_load(A, b, Q)
            st, r, eh, ah = F.fftm_solve_step(gp.p, history_len=wl.max_iter + 1)
            assert r["converged"], (k, r)
            Sg = gp.get_voxel(F.FFTM_FIELD_STRESS)
            Gg = gp.get_voxel(F.FFTM_FIELD_GRAD)
            if precision == "fp64":
                assert r["iterations"] == rep.iterations, (k, r["iterations"], rep.iterations)
                assert [i for i, a in enumerate(ah) if a] == rep.accelerated
                tol = 1e-9
            else:
                # FP32 follows the oracle's error history to ~1e-5; below that the residual's
                # rounding floor (~1.4e-7 here, 7x under the tolerance) makes the Anderson steps
                # slightly less effective and the crossing of tol can move by one Anderson period
                assert abs(r["iterations"] - rep.iterations) <= 3, (k, r["iterations"], rep.iterations)
                tol = 1e-5
            assert rel_l2(Sg, _s9(pr.last["P"])) < tol, k
            assert rel_l2(Gg, pr.last["G"].reshape(Gg.shape)) < tol, k
    finally:
        gp.close()


# ---- FCC crystal plasticity (Sec. 3.4), torsion-bending of a small polycrystal ------------
CP_PARAMS = (168.0, 121.0, 75.0, 1e-3, 20.0, 0.03, 0.09, 0.3, 1.0)  # C11 C12 C44 gdot0 n tau0 tau_inf h0 dt


def _cp(tol):
    n = (8, 6, 6)
    ph, _ = syn.voronoi(n, 4, 5)
    quats = syn.shoemake_quaternions(4, 6)
    mats = [Material(syn.workloads.CP_FCC, CP_PARAMS, tuple(q)) for q in quats]
    wl = Workload("cp_tb", n, ph, mats, axis_bc("D", "N", "N"), scheme="TETRA2", lambda0=121.0, mu0=49.25,
                  tol=tol, max_iter=3000)
    loads = [syn.torsion_bending_load(n, (1.0, 1.0, 1.0), k * 0.05 / 4, k * 0.02 / 4) for k in (1, 2)]
    return wl, loads


def _fp_state(st):
    """oracle (F^p, Gamma) -> (npp, 10, n1, n2, n3), F^p row-major."""
    Fp = st["Fp"]
    return np.concatenate([Fp.reshape(Fp.shape[0], 9, *Fp.shape[3:]), st["gam"][:, None]], axis=1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_crystal_plasticity_torsion_bending_matches_the_oracle(precision):
    wl, loads = _cp(1e-8 if precision == "fp64" else 1e-6)
    pr = Problem(wl)
    gp = GpuProblem(wl, precision)
    try:
        slipped = False
        for k, (A, b, Q) in enumerate(loads):
            _, rep = pr.solve_step(A=A, b=b, Q=Q)
            assert rep.converged
            gp.set_load(A, b, Q)
            st, r, eh, ah = F.fftm_solve_step(gp.p, history_len=wl.max_iter + 1)
            assert r["converged"], (k, r)
            Sg = gp.get_voxel(F.FFTM_FIELD_STRESS)
            Zg = gp.get_voxel(F.FFTM_FIELD_STATE)
            Zo = _fp_state(pr.state)
            slipped |= Zo[:, 9].max() > 1e-3
            if precision == "fp64":
                # hundreds of iterations: allow the count to move by one Anderson period; the
                # fields agree to the fixed point's tolerance (1e-8) times its conditioning
                assert abs(r["iterations"] - rep.iterations) <= 3, (k, r["iterations"], rep.iterations)
                assert rel_l2(Sg, _s9(pr.last["P"])) < 1e-7, k
                assert rel_l2(Zg, Zo) < 1e-7, k
            else:
                # fields to the 1e-5 bar; the iteration count is not held to +-2: the FP32 residual
                # of this quasi rate-independent law floors near 1e-6 (the law's Newton rounds at
                # ~1e-7 of the stress and the soft plastic tangent amplifies it), so FP32 tracks
                # the oracle's error history to ~1e-4 and then needs 2-3x the iterations to
                # cross 1e-6
                assert rel_l2(Sg, _s9(pr.last["P"])) < 1e-5, k
                assert rel_l2(Zg, Zo) < 1e-5, k
                assert rep.iterations - 3 <= r["iterations"] <= 4 * rep.iterations, (k, r["iterations"],
                                                                                       rep.iterations)
        assert slipped, "the load must take the crystals well into slip"
    finally:
        gp.close()
