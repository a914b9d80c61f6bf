"""Non-zero Neumann tractions (Sec. 2.2, P* = 2 t at the mirror voxel centres) on the GPU.

* The end-loaded homogeneous bar lands on its uniaxial-stress closed form (FP64 and FP32,
  HEX1 and TETRA2).
* A two-phase medium with a traction-loaded end reproduces the oracle: FP64 with its
  iteration count, Anderson steps and stress field to 1e-9; FP32 within +-2 iterations and
  1e-5.
* A J2 matrix loaded by traction over two steps (the second past yield) goes through the
  incremental residual, which takes only the traction's change since the commit: FP64
  matches the oracle's iterations and stresses at both steps.
* Non-uniform tractions on a face (smooth normal and shear fields over the face's voxels)
  reproduce the oracle's stencils.add_traction_ghosts construction: FP64 with
  its iteration count and stresses to 1e-9, FP32 within +-2 iterations and 1e-5; the field
  on a J2 matrix over two steps goes through the incremental residual (its change since the
  commit) with the oracle's iterations.
* A traction on a component that is not Neumann on that face is refused, uniform or field.
"""

import numpy as np
import pytest

import synthetic as syn
from abi_helpers import GpuProblem, rel_l2, sym6
from oracle.solver import Problem
from paper_2607_05929_gb300 import build
from paper_2607_05929_gb300 import fftm as F
from synthetic.workloads import ISO_ELASTIC, J2_LINHARD, Material, Workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    F.load_library()


def _bar_bc():
    # component 1 Dirichlet on the x = 0 face only; everything else Neumann
    return [[["D", "N", "N"], ["N", "N", "N"]], [["N"] * 3, ["N"] * 3], [["N"] * 3, ["N"] * 3]]


def _end_traction(t1, t2=0.0):
    T = np.zeros((3, 2, 3))
    T[0, 1, 0] = t1
    T[0, 1, 1] = t2
    return T


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_end_loaded_bar_on_the_gpu_is_in_uniaxial_stress(scheme, precision):
    E, nu, sig = 2.0, 0.3, 1e-3
    lam, mu = syn.iso_lame(E, nu)
    n = (8, 6, 6)
    tol = 1e-12 if precision == "fp64" else 1e-6
    wl = Workload("bar_traction", n, np.zeros(n, np.uint16), [Material(ISO_ELASTIC, (lam, mu))], _bar_bc(),
                  scheme=scheme, lambda0=lam, mu0=mu, tol=tol, A=np.zeros((3, 3)), max_iter=3000)
    gp = GpuProblem(wl, precision)
    try:
        gp.set_load(np.zeros((3, 3)), np.zeros(3), np.zeros((3, 6)), T=_end_traction(sig))
        st, r, _, _ = F.fftm_solve_step(gp.p)
        assert st == F.FFTM_OK and r["converged"]
        bar = 1e-10 if precision == "fp64" else 1e-5
        S = gp.get_voxel(F.FFTM_FIELD_STRESS)  # (npp, 6, n1, n2, n3): 11, 22, 33, 23, 13, 12
        expect = np.array([sig, 0, 0, 0, 0, 0])[None, :, None, None, None]
        assert np.abs(S - expect).max() < bar * sig
        G = gp.get_voxel(F.FFTM_FIELD_GRAD)
        G = G.reshape(G.shape[0], 3, 3, *G.shape[2:])
        eps = 0.5 * (G + np.swapaxes(G, 1, 2))
        e = np.diag([sig / E, -nu * sig / E, -nu * sig / E])[None, :, :, None, None, None]
        assert np.abs(eps - e).max() < bar * sig / E
    finally:
        gp.close()


def _block_bc():
    # the bar's x faces; on the y and z faces the normal component is held (Dirichlet) and
    # the tangential ones are free, which removes the rigid rotation about x that the bar's
    # all-free lateral faces leave (a zero-energy mode that rounding excites differently in
    # every implementation and that makes iteration counts drift)
    return [[["D", "N", "N"], ["N", "N", "N"]], [["N", "D", "N"], ["N", "D", "N"]], [["N", "N", "D"], ["N", "N", "D"]]]


def _two_phase(scheme, tol, law=ISO_ELASTIC):
    n = (12, 9, 8)
    lam1, mu1 = syn.iso_lame(1.0, 0.3)
    lam2, mu2 = syn.iso_lame(6.0, 0.25)
    ph = syn.random_spheres(n, 0.25, 1.5, 2.5, 12)
    m1 = Material(J2_LINHARD, (lam1, mu1, 4e-4, 0.05)) if law == J2_LINHARD else Material(ISO_ELASTIC, (lam1, mu1))
    mats = [m1, Material(ISO_ELASTIC, (lam2, mu2))]
    return Workload("traction_2ph", n, ph, mats, _block_bc(), scheme=scheme, lambda0=0.5 * (lam1 + lam2),
                    mu0=0.5 * (mu1 + mu2), tol=tol, A=np.zeros((3, 3)), max_iter=3000)


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_traction_two_phase_fp64_matches_the_oracle(scheme):
    wl = _two_phase(scheme, 1e-10)
    T = _end_traction(1e-3)
    pr = Problem(wl)
    uf, rep = pr.solve_step(T=T)
    assert rep.converged
    gp = GpuProblem(wl, "fp64")
    try:
        gp.set_load(np.zeros((3, 3)), np.zeros(3), np.zeros((3, 6)), T=T)
        st, r, eh, ah = F.fftm_solve_step(gp.p, history_len=wl.max_iter + 1)
        assert st == F.FFTM_OK and r["converged"]
        assert r["iterations"] == rep.iterations, (r["iterations"], rep.iterations)
        assert [i for i, a in enumerate(ah) if a] == rep.accelerated
        assert rel_l2(gp.get_voxel(F.FFTM_FIELD_STRESS), sym6(pr.last["P"])) < 1e-9
    finally:
        gp.close()


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_traction_two_phase_fp32_vs_fp64_oracle(scheme):
    wl = _two_phase(scheme, 1e-6)
    T = _end_traction(1e-3)
    pr = Problem(wl)
    uf, rep = pr.solve_step(T=T)
    assert rep.converged
    gp = GpuProblem(wl, "fp32")
    try:
        gp.set_load(np.zeros((3, 3)), np.zeros(3), np.zeros((3, 6)), T=T)
        st, r, _, _ = F.fftm_solve_step(gp.p)
        assert r["converged"]
        assert abs(r["iterations"] - rep.iterations) <= 2, (r["iterations"], rep.iterations)
        assert rel_l2(gp.get_voxel(F.FFTM_FIELD_STRESS), sym6(pr.last["P"])) < 1e-5
    finally:
        gp.close()


def test_traction_j2_two_steps_through_the_incremental_residual():
    wl = _two_phase("HEX1", 1e-10, law=J2_LINHARD)
    pr = Problem(wl)
    gp = GpuProblem(wl, "fp64")
    try:
        yielded = False
        for t in (3e-4, 6e-4):
            T = _end_traction(t)
            _, rep = pr.solve_step(T=T)
            assert rep.converged
            gp.set_load(np.zeros((3, 3)), np.zeros(3), np.zeros((3, 6)), T=T)
            st, r, _, _ = F.fftm_solve_step(gp.p, history_len=wl.max_iter + 1)
            assert st == F.FFTM_OK and r["converged"]
            assert r["iterations"] == rep.iterations, (t, r["iterations"], rep.iterations)
            assert rel_l2(gp.get_voxel(F.FFTM_FIELD_STRESS), sym6(pr.last["P"])) < 1e-9
            yielded = yielded or float(np.abs(pr.state["p"]).max()) > 0.0
        assert yielded, "the second step must take the matrix past yield"
    finally:
        gp.close()


def test_traction_on_a_dirichlet_component_is_refused():
    lam, mu = syn.iso_lame(1.0, 0.3)
    n = (8, 6, 6)
    wl = Workload("bad_traction", n, np.zeros(n, np.uint16), [Material(ISO_ELASTIC, (lam, mu))], _bar_bc(),
                  scheme="HEX1", lambda0=lam, mu0=mu, tol=1e-8, A=np.zeros((3, 3)))
    gp = GpuProblem(wl, "fp64")
    try:
        T = np.zeros((3, 2, 3))
        T[0, 0, 0] = 1e-3  # component 1 is Dirichlet on the x = 0 face
        with pytest.raises(F.FFTMError):
            gp.set_load(np.zeros((3, 3)), np.zeros(3), np.zeros((3, 6)), T=T)
    finally:
        gp.close()


def _face_field(n, seed, scale):
    """(3, n_y, n_z) field over the x = L face (oracle order [q][b][c] with b = y, c = z) and its
    ABI array (3, n_z, n_y): a normal load and a shear load, both varying over the face (phases
    drawn from the seed), component 3 zero."""
    rng = np.random.default_rng(seed)
    y = (np.arange(n[1]) + 0.5) / n[1]
    z = (np.arange(n[2]) + 0.5) / n[2]
    ph = rng.uniform(0.0, np.pi, 2)
    t = np.zeros((3, n[1], n[2]))
    t[0] = scale * (1.0 + 0.5 * np.outer(np.sin(np.pi * y + ph[0]), np.cos(np.pi * z)))
    t[1] = 0.2 * scale * np.outer(np.cos(2 * np.pi * y + ph[1]), np.sin(np.pi * z))
    return t, np.ascontiguousarray(t.transpose(0, 2, 1))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_face_traction_field_matches_the_oracle(scheme, precision):
    wl = _two_phase(scheme, 1e-10 if precision == "fp64" else 1e-6)
    t, t_abi = _face_field(wl.n, 13, 1e-3)
    pr = Problem(wl)
    uf, rep = pr.solve_step(Tf={(0, 1): t})
    assert rep.converged
    gp = GpuProblem(wl, precision)
    try:
        F.fftm_set_face_traction(gp.p, 0, 1, t_abi.astype(gp.dtype))
        st, r, eh, ah = F.fftm_solve_step(gp.p, history_len=wl.max_iter + 1)
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


def test_face_traction_field_j2_two_steps_through_the_incremental_residual():
    wl = _two_phase("HEX1", 1e-10, law=J2_LINHARD)
    pr = Problem(wl)
    gp = GpuProblem(wl, "fp64")
    try:
        for k, scale in enumerate((3e-4, 6e-4)):
            t, t_abi = _face_field(wl.n, 14, scale)
            _, rep = pr.solve_step(Tf={(0, 1): t})
            assert rep.converged
            F.fftm_set_face_traction(gp.p, 0, 1, t_abi)
            st, r, _, _ = F.fftm_solve_step(gp.p, history_len=wl.max_iter + 1)
            assert st == F.FFTM_OK and r["converged"]
            assert r["iterations"] == rep.iterations, (k, r["iterations"], rep.iterations)
            assert rel_l2(gp.get_voxel(F.FFTM_FIELD_STRESS), sym6(pr.last["P"])) < 1e-9
    finally:
        gp.close()


def test_face_traction_field_on_a_dirichlet_component_is_refused():
    wl = _two_phase("HEX1", 1e-8)
    gp = GpuProblem(wl, "fp64")
    try:
        bad = np.zeros((3, wl.n[1], wl.n[2]))
        bad[0] = 1e-3  # component 1 is Dirichlet on the x = 0 face
        with pytest.raises(F.FFTMError):
            F.fftm_set_face_traction(gp.p, 0, 0, bad)
        with pytest.raises(F.FFTMError):
            F.fftm_set_face_traction(gp.p, 0, 1, np.zeros((3, 2, 2)))  # wrong size
    finally:
        gp.close()
