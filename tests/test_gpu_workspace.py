"""A problem built inside a caller's device workspace (fftm_problem_create_in), here a torch
tensor: no device memory is taken outside it while the problem is created and solved, and the
load step is bit-identical to the one of a problem that allocates its own memory; a workspace
below fftm_problem_workspace_bytes or misaligned is refused."""

import numpy as np
import pytest

import synthetic as syn
from paper_2607_05929_gb300 import build
from paper_2607_05929_gb300 import fftm as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    F.load_library()


def _desc(wl, precision):
    mats = [(m.law, m.params, m.quat) for m in wl.materials]
    return F.make_desc(wl.n, wl.phase, mats, wl.bc, scheme=wl.scheme, green=wl.green, lambda0=wl.lambda0,
                       mu0=wl.mu0, precision=precision, tol=1e-8 if precision == "fp64" else 1e-6,
                       max_iter=wl.max_iter)


@pytest.mark.parametrize("precision", ["fp64", "fp32_tf32"])
def test_problem_in_a_torch_workspace(precision):
    torch = pytest.importorskip("torch")
    wl = syn.voronoi_polycrystal(n=(64, 48, 32), grains=12)
    ctx = F.fftm_ctx_create(0, None)
    runs = []
    try:
        for inside in (True, False):
            desc, keep = _desc(wl, precision)
            need = F.fftm_problem_workspace_bytes(desc)
            ws = torch.empty(need, dtype=torch.uint8, device="cuda") if inside else None
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            p = F.fftm_problem_create_in(ctx, desc, ws) if inside else F.fftm_problem_create(ctx, desc)
            try:
                F.fftm_set_load(p, wl.A)
                st, r, eh, ah = F.fftm_solve_step(p, history_len=wl.max_iter + 1)
                torch.cuda.synchronize()
                taken = free0 - torch.cuda.mem_get_info()[0]
                N = F.fftm_problem_layout(p)[0]
                u = np.zeros((3, N[2], N[1], N[0]), dtype=np.float64 if precision == "fp64" else np.float32)
                F.fftm_get_field(p, F.FFTM_FIELD_U, u)
                runs.append((r, eh, u, taken, need))
            finally:
                F.fftm_problem_destroy(p)
            del ws
    finally:
        F.fftm_ctx_destroy(ctx)
    (r1, e1, u1, taken1, need), (r2, e2, u2, taken2, _) = runs
    assert r1["converged"] and r1["iterations"] == r2["iterations"]
    assert np.array_equal(e1, e2) and np.array_equal(u1, u2)
    # the workspace problem took (almost) no device memory of its own; the other one took it all
    assert taken1 < 0.05 * need, (taken1, need)
    assert taken2 > 0.5 * need, (taken2, need)


def test_a_small_or_misaligned_workspace_is_refused():
    torch = pytest.importorskip("torch")
    wl = syn.voronoi_polycrystal(n=(32, 24, 16), grains=6)
    ctx = F.fftm_ctx_create(0, None)
    try:
        desc, keep = _desc(wl, "fp32")
        need = F.fftm_problem_workspace_bytes(desc)
        ws = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
        with pytest.raises(F.FFTMError) as e:
            F.fftm_problem_create_in(ctx, desc, ws[: need - 256])
        assert e.value.status == F.FFTM_E_NOMEM
        with pytest.raises(F.FFTMError) as e:
            F.fftm_problem_create_in(ctx, desc, ws[16: need + 16])
        assert e.value.status == F.FFTM_E_INVALID
    finally:
        F.fftm_ctx_destroy(ctx)
