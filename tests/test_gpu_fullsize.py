"""The 256^3 polycrystal the bench times, solved by the precision form (FP32 fields with TF32
transform contractions, the launch configuration of the bench), checked by the FP64 oracle at full
size: the oracle's own residual of the GPU's converged displacement (u^f read as its high and low
parts) meets the load step's tolerance, the GPU's equilibrium error and mean stress agree with the
oracle's evaluation of the same field, and the GPU's residual field D matches the oracle's on that
field.  The oracle evaluates one residual of the whole grid (about a minute on the host cores)."""

import numpy as np
import pytest

import bench
from abi_helpers import node_from_abi, rel_l2
from oracle.solver import Problem
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
    # agrees with it to the FP32 residual's rounding (a few 1e-8 of the stress scale, i.e. a few
    # per cent of D when err is 1e-6)
    assert err < 1.1 * wl.tol, (err, r["err"])
    assert abs(err - r["err"]) <= 0.1 * err, (err, r["err"])
    assert rel_l2(node_from_abi(Dg.astype(np.float64)), D_ref) < 0.1
    Pm = P_ref.mean(axis=(0, 3, 4, 5))
    ref = np.array([Pm[0, 0], Pm[1, 1], Pm[2, 2], Pm[1, 2], Pm[0, 2], Pm[0, 1]])
    assert np.linalg.norm(r["mean_P"] - ref) <= 1e-5 * np.linalg.norm(ref)
