"""fftm_residual_noalloc agrees with the regular residual entry point (FFTM_OP_RESIDUAL).

Callers that may not allocate device memory where they need a residual --
inside CUDA stream capture, under a framework that owns every device byte
through its own pool, in fixed-memory real-time loops -- pass their own u, D
and norm buffers to fftm_residual_noalloc, whose reduction partials live in a
static device array of the library.  Two calls in a row must both reproduce
the regular entry point's D and norms, to the tolerance of the other GPU
parity tests.
"""

import numpy as np
import pytest

import synthetic as syn
from abi_helpers import GpuProblem, node_from_abi, node_to_abi, rel_l2, sym6
from paper_2607_05929_gb300 import build
from paper_2607_05929_gb300 import fftm as F
from synthetic.workloads import CUBIC_ELASTIC, Material, Workload, axis_bc

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 2e-5}


def _workload():
    n = (24, 18, 16)
    ph, _ = syn.voronoi(n, 5, 3)
    q = syn.shoemake_quaternions(5, 4)
    mats = [Material(CUBIC_ELASTIC, (168.0, 121.0, 75.0), tuple(v)) for v in q]
    A = np.zeros((3, 3))
    A[0, 0] = 1e-3
    A[2, 1] = -4e-4
    return Workload("noalloc", n, ph, mats, axis_bc("D", "N", "P"), scheme="TETRA2", lambda0=121.0,
                    mu0=49.25, tol=1e-6, A=A)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_residual_matches_the_regular_entry_point_on_two_calls(precision):
    build.build()
    F.load_library()
    wl = _workload()
    gp = GpuProblem(wl, precision)
    try:
        rng = np.random.default_rng(17)
        N = gp.N
        u = 1e-3 * rng.standard_normal((3,) + N)
        u[:, 0] = 0.0  # Dirichlet x faces: u^f vanishes there
        u[:, -1] = 0.0
        gp.set_node(F.FFTM_FIELD_U, u)
        _, norms_ref = F.fftm_apply(gp.p, F.FFTM_OP_RESIDUAL)
        D_ref = gp.get_node(F.FFTM_FIELD_D)

        tdt = torch.float64 if precision == "fp64" else torch.float32
        u_dev = torch.from_numpy(node_to_abi(u).astype(gp.dtype)).cuda()
        for call in range(2):
            D_dev = torch.full(u_dev.shape, float("nan"), dtype=tdt, device="cuda")
            norms_dev = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            F.fftm_residual_noalloc(gp.p, u_dev, D_dev, norms_dev)
            torch.cuda.synchronize()
            D = node_from_abi(D_dev.cpu().numpy()).astype(np.float64)
            norms = norms_dev.cpu().numpy()
            assert np.isfinite(D).all(), f"call {call}: D not fully written"
            assert rel_l2(D, D_ref) < TOL[precision], call
            assert np.allclose(norms, norms_ref, rtol=TOL[precision], atol=0.0), (call, norms, norms_ref)
    finally:
        gp.close()


def _j2_bending():
    wl, loads = syn.sphere_composite_bending((12, 9, 8), r_min=2.0, r_max=3.0, seed=4, scheme="HEX1", steps=20,
                                             theta_max=0.012 * 12 / 9, tol=1e-8)
    return wl, loads[:8]  # the last steps take the matrix past yield: a committed plastic state


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["cubic", "j2_after_commits"])
def test_noalloc_residual_matches_the_oracle(precision, case):
    """D and the norms of fftm_residual_noalloc against the FP64 oracle's residual (a1-a4), on
    a cubic polycrystal and on a J2 composite after eight committed bending steps (past yield):
    the entry point evaluates the residual in the plain form from the committed state, the
    solver after a commit in the incremental one; both must equal the oracle's D."""
    from oracle.solver import Problem

    build.build()
    F.load_library()
    if case == "cubic":
        wl, loads = _workload(), []
    else:
        wl, loads = _j2_bending()
    pr = Problem(wl)
    gp = GpuProblem(wl, precision, tol=1e-8 if precision == "fp64" else 1e-6)
    try:
        for A, b, Q in loads:
            _, rep = pr.solve_step(A=A, b=b, Q=Q)
            assert rep.converged
            gp.set_load(A, b, Q)
            st, r, _, _ = F.fftm_solve_step(gp.p)
            assert r["converged"]
        if loads:
            assert float(np.abs(pr.state["p"]).max()) > 0.0, "the schedule should reach yield"
            # the oracle's committed plastic state, so that D depends on the same state on both sides
            st6 = np.concatenate([sym6(pr.state["ep"]), pr.state["p"][:, None]], axis=1)
            F.fftm_set_field(gp.p, F.FFTM_FIELD_STATE,
                             np.ascontiguousarray(st6.transpose(0, 1, 4, 3, 2)).astype(gp.dtype).ravel())
            Gs = pr.grad_ustar(*loads[-1])
        else:
            Gs = pr.grad_ustar()
        rng = np.random.default_rng(23)
        u = pr.uf + 1e-2 * np.abs(pr.uf).max() * rng.standard_normal(pr.grid.node_shape) if loads else \
            1e-3 * rng.standard_normal(pr.grid.node_shape)
        for q in range(3):
            u[q][~pr.grid.dof_mask(q)] = 0.0
        u = u.astype(gp.dtype).astype(np.float64)  # the field the library receives
        _, D_ref, _, _, SD, SP = pr.residual(u, Gs)
        tdt = torch.float64 if precision == "fp64" else torch.float32
        u_dev = torch.from_numpy(node_to_abi(u).astype(gp.dtype)).cuda()
        D_dev = torch.full(u_dev.shape, float("nan"), dtype=tdt, device="cuda")
        norms_dev = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        F.fftm_residual_noalloc(gp.p, u_dev, D_dev, norms_dev)
        torch.cuda.synchronize()
        D = node_from_abi(D_dev.cpu().numpy()).astype(np.float64)
        norms = norms_dev.cpu().numpy()
        tol = TOL[precision]
        assert rel_l2(D, D_ref) < tol
        assert abs(norms[0] - SD) < 10 * tol * SD and abs(norms[1] - SP) < tol * SP
    finally:
        gp.close()
