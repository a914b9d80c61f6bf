"""u* given as a node field (fftm_set_load_field) on the GPU against the oracle, through the
C ABI:

* the closed-form affine-plus-quadratic load and the same displacement given as node values
  give the same FP64 load step (iterations, stresses to 1e-12), both schemes;
* a smooth field that is not a polynomial, added to an affine load on a two-phase medium:
  FP64 with the oracle's iteration count and stresses to 1e-9; FP32 (FFT and TF32 transforms)
  within +-2 iterations and 1e-5;
* a J2 matrix under a growing field over two steps goes through the incremental residual (the
  field's change since the commit) with the oracle's iteration counts and stresses to 1e-9.
"""

import numpy as np
import pytest

import synthetic as syn
from abi_helpers import GpuProblem, node_to_abi, rel_l2, sym6
from oracle.solver import Problem
from paper_2607_05929_gb300 import build
from paper_2607_05929_gb300 import fftm as F
from synthetic.workloads import ISO_ELASTIC, J2_LINHARD, Material, Workload, axis_bc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    F.load_library()


def _wl(scheme, tol, law=ISO_ELASTIC):
    n = (12, 9, 8)
    lam1, mu1 = syn.iso_lame(1.0, 0.3)
    lam2, mu2 = syn.iso_lame(4.0, 0.25)
    ph = syn.random_spheres(n, 0.2, 1.5, 2.0, 9)
    m1 = Material(J2_LINHARD, (lam1, mu1, 5e-4, 0.05)) if law == J2_LINHARD else Material(ISO_ELASTIC, (lam1, mu1))
    return Workload("ustar_field", n, ph, [m1, Material(ISO_ELASTIC, (lam2, mu2))], axis_bc("D", "N", "N"),
                    scheme=scheme, lambda0=0.5 * (lam1 + lam2), mu0=0.5 * (mu1 + mu2), tol=tol, max_iter=3000)


def _field(pr, scale):
    g = pr.grid
    X = np.meshgrid(*[np.arange(g.N[a]) * g.h[a] for a in range(3)], indexing="ij")
    L = [g.n[a] * g.h[a] for a in range(3)]
    bump = np.sin(np.pi * X[0] / L[0]) * (1.0 + X[1] / L[1]) * np.cos(X[2] / L[2])
    shear = X[0] / L[0] * np.sin(2 * np.pi * X[1] / L[1])  # non-zero on the x = L face
    return scale * np.stack([bump + shear, 0.5 * bump, -bump + 0.3 * shear])


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_closed_form_and_node_field_agree(scheme):
    wl = _wl(scheme, 1e-10)
    rng = np.random.default_rng(2)
    A = 1e-3 * rng.standard_normal((3, 3))
    Q = 1e-4 * rng.standard_normal((3, 6))
    pr = Problem(wl)
    X = np.meshgrid(*[np.arange(pr.grid.N[a]) * pr.grid.h[a] for a in range(3)], indexing="ij")
    mono = [X[0] * X[0], X[1] * X[1], X[2] * X[2], X[1] * X[2], X[0] * X[2], X[0] * X[1]]
    Us = np.stack([sum(A[q, a] * X[a] for a in range(3)) + sum(Q[q, k] * mono[k] for k in range(6))
                   for q in range(3)])
    out = []
    for field in (False, True):
        gp = GpuProblem(wl, "fp64")
        try:
            if field:
                gp.set_load(np.zeros((3, 3)), np.zeros(3), np.zeros((3, 6)))
                F.fftm_set_load_field(gp.p, node_to_abi(Us))
            else:
                gp.set_load(A, np.zeros(3), Q)
            st, r, _, _ = F.fftm_solve_step(gp.p, history_len=wl.max_iter + 1)
            assert r["converged"]
            out.append((r["iterations"], gp.get_voxel(F.FFTM_FIELD_STRESS)))
        finally:
            gp.close()
    assert out[0][0] == out[1][0]
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-12 * np.abs(out[0][1]).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_tf32"])
@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_smooth_field_matches_the_oracle(scheme, precision):
    wl = _wl(scheme, 1e-10 if precision == "fp64" else 1e-6)
    A = np.zeros((3, 3))
    A[0, 0] = 1e-3
    pr = Problem(wl)
    Us = _field(pr, 1e-3)
    _, rep = pr.solve_step(A=A, Us=Us)
    assert rep.converged
    gp = GpuProblem(wl, precision)
    try:
        gp.set_load(A, np.zeros(3), np.zeros((3, 6)))
        F.fftm_set_load_field(gp.p, node_to_abi(Us).astype(gp.dtype))
        st, r, _, _ = F.fftm_solve_step(gp.p, history_len=wl.max_iter + 1)
        assert r["converged"], r
        S = gp.get_voxel(F.FFTM_FIELD_STRESS)
        if precision == "fp64":
            assert r["iterations"] == rep.iterations, (r["iterations"], rep.iterations)
            assert rel_l2(S, sym6(pr.last["P"])) < 1e-9
        else:
            assert abs(r["iterations"] - rep.iterations) <= 2, (r["iterations"], rep.iterations)
            assert rel_l2(S, sym6(pr.last["P"])) < 1e-5
    finally:
        gp.close()


def test_growing_field_on_j2_goes_through_the_incremental_residual():
    wl = _wl("HEX1", 1e-10, law=J2_LINHARD)
    pr = Problem(wl)
    gp = GpuProblem(wl, "fp64")
    try:
        yielded = False
        for scale in (1e-3, 2.5e-3):
            A = np.zeros((3, 3))
            A[0, 0] = scale
            Us = _field(pr, scale)
            _, rep = pr.solve_step(A=A, Us=Us)
            assert rep.converged
            gp.set_load(A, np.zeros(3), np.zeros((3, 6)))
            F.fftm_set_load_field(gp.p, node_to_abi(Us))
            st, r, _, _ = F.fftm_solve_step(gp.p, history_len=wl.max_iter + 1)
            assert st == F.FFTM_OK and r["converged"]
            assert r["iterations"] == rep.iterations, (scale, r["iterations"], rep.iterations)
            assert rel_l2(gp.get_voxel(F.FFTM_FIELD_STRESS), sym6(pr.last["P"])) < 1e-9
            yielded = yielded or float(np.abs(pr.state["p"]).max()) > 0.0
        assert yielded, "the second step must take the matrix past yield"
    finally:
        gp.close()
