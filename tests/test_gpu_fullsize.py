"""The 256^3 polycrystal the bench times, solved by the precision form (FP32 fields with TF32
transform contractions, the launch configuration of the bench), checked by the FP64 oracle at full
size: the oracle's own residual of the GPU's converged displacement (u^f read as its high and low
parts) meets the load step's tolerance, the GPU's equilibrium error and mean stress agree with the
oracle's evaluation of the same field, and the GPU's residual field D differs from the oracle's by
no more than FP32 rounding accounts for.  At convergence D is about 1e-6 of the stress scale, so the
FP32 evaluation of the stresses (rounding of a few units of 2^-24 on each entry, summed with
cancellation by the divergence) is a visible fraction of D: the bound is stated against the
divergence of the oracle's stress rounded once to FP32, times the number of roundings a stress entry
and a node's sum go through on the GPU.  The oracle evaluates one residual of the whole grid."""

import numpy as np
import pytest

import bench
from abi_helpers import node_from_abi, rel_l2
from oracle.solver import Problem
from oracle.stencils import div
from paper_2607_05929_gb300 import build
from paper_2607_05929_gb300 import fftm as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    F.load_library()


def test_full_size_tf32_solve_is_an_equilibrium_of_the_oracle():
    wl = bench.workload(256, 500)
    ctx = F.fftm_ctx_create(0, None)
    mats = [(m.law, m.params, m.quat) for m in wl.materials]
    desc, keep = F.make_desc(wl.n, wl.phase, mats, wl.bc, scheme=wl.scheme, green=wl.green, lambda0=wl.lambda0,
                             mu0=wl.mu0, precision="fp32_tf32", tol=wl.tol, max_iter=wl.max_iter)
    p = F.fftm_problem_create(ctx, desc)
    try:
        F.fftm_set_load(p, wl.A)
        st, r, eh, ah = F.fftm_solve_step(p, history_len=wl.max_iter + 1)
        assert r["converged"], r
        N = F.fftm_problem_layout(p)[0]
        hi = np.zeros((3, N[2], N[1], N[0]), dtype=np.float32)
        lo = np.zeros_like(hi)
        F.fftm_get_field(p, F.FFTM_FIELD_U, hi)
        F.fftm_get_field(p, F.FFTM_FIELD_U_LO, lo)
        _, norms = F.fftm_apply(p, F.FFTM_OP_RESIDUAL)
        Dg = np.zeros((3, N[2], N[1], N[0]), dtype=np.float32)
        F.fftm_get_field(p, F.FFTM_FIELD_D, Dg)
    finally:
        F.fftm_problem_destroy(p)
        F.fftm_ctx_destroy(ctx)
    u = node_from_abi(hi.astype(np.float64) + lo.astype(np.float64))
    pr = Problem(wl)
    p_ref, D_ref, P_ref, G_ref, SD, SP = pr.residual(u, pr.grad_ustar())
    err = pr.error(SD, SP)
    # the GPU stopped at its FP32 evaluation of err < tol; the FP64 evaluation of the same field
    # agrees with it to the FP32 residual's rounding, which adds in quadrature to D
    assert err < 1.1 * wl.tol, (err, r["err"])
    assert abs(err - r["err"]) <= 0.1 * err, (err, r["err"])
    # rounding model: the divergence of one FP32 rounding of every stress entry; the GPU rounds the
    # gradient, each term of the law and each partial sum of a node's divergence, so its deviation
    # is a small multiple of the model (16 bounds the gradient + law + sum chain with margin)
    dP = P_ref.astype(np.float32).astype(np.float64) - P_ref
    D_round = div(dP, pr.grid, pr.scheme)
    for q in range(3):
        D_round[q][~pr.masks[q]] = 0.0
    dev = float(np.linalg.norm(node_from_abi(Dg.astype(np.float64)) - D_ref))
    model = float(np.linalg.norm(D_round))
    print(f"|D_gpu - D_ref| = {dev:.3e}, one-rounding model {model:.3e}, ratio {dev / model:.2f}, "
          f"|D_ref| = {np.linalg.norm(D_ref):.3e}")
    assert dev <= 16.0 * model, (dev, model)
    Pm = P_ref.mean(axis=(0, 3, 4, 5))
    ref = np.array([Pm[0, 0], Pm[1, 1], Pm[2, 2], Pm[1, 2], Pm[0, 2], Pm[0, 1]])
    assert np.linalg.norm(r["mean_P"] - ref) <= 1e-5 * np.linalg.norm(ref)
