"""Descriptor checks of the logarithmic J2 law on the host (no GPU): the library refuses
invalid parameters and a second law with internal variables in the same problem, and
counts the committed and next state in the workspace estimate."""

import numpy as np
import pytest

from paper_2607_05929_gb300 import build
from paper_2607_05929_gb300 import fftm as F
from paper_2607_05929_gb300 import fftm as Fm
from synthetic.workloads import ISO_ELASTIC, J2_LINHARD, LOG_J2, NEO_HOOKE

LAM, MU, SIG0 = 1.2, 0.8, 2e-3
Q1 = (1.0, 0.0, 0.0, 0.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    F.load_library()


def _desc(mats, precision="fp64"):
    n = (6, 4, 4)
    ph = np.zeros(n, np.uint16)
    ph[2:4, 1:3, 1:3] = 1
    bc = [[["D"] * 3] * 2, [["N"] * 3] * 2, [["N"] * 3] * 2]
    return F.make_desc(n, ph, mats, bc, scheme="TETRA2", lambda0=LAM, mu0=MU, precision=precision, tol=1e-8,
                       max_iter=100)


@pytest.mark.parametrize("params", [(LAM, 0.0, SIG0), (LAM, MU, 0.0), (-MU, MU, SIG0)])
def test_invalid_parameters_are_refused(params):
    desc, keep = _desc([(LOG_J2, params, Q1), (NEO_HOOKE, (0.05, 0.1), Q1)])
    with pytest.raises(F.FFTMError) as e:
        F.fftm_problem_workspace_bytes(desc)
    assert e.value.status == F.FFTM_E_INVALID


def test_a_second_law_with_internal_variables_is_refused():
    desc, keep = _desc([(LOG_J2, (LAM, MU, SIG0), Q1), (J2_LINHARD, (LAM, MU, SIG0, 0.0), Q1)])
    with pytest.raises(F.FFTMError) as e:
        F.fftm_problem_workspace_bytes(desc)
    assert e.value.status == F.FFTM_E_UNSUPPORTED


def test_workspace_counts_both_state_buffers():
    el, keep = _desc([(ISO_ELASTIC, (LAM, MU), Q1), (NEO_HOOKE, (0.05, 0.1), Q1)])
    lj, keep2 = _desc([(LOG_J2, (LAM, MU, SIG0), Q1), (NEO_HOOKE, (0.05, 0.1), Q1)])
    npp, nvox = 2, 6 * 4 * 4
    assert F.fftm_problem_workspace_bytes(lj) - F.fftm_problem_workspace_bytes(el) == 2 * npp * 7 * nvox * 8


def _G_of_F(F):
    return (F - np.eye(3)).T


@pytest.mark.parametrize("seed", range(6))
def test_the_library_law_matches_the_oracle_pointwise(seed):
    """The library's law code (run on the host, FP64) against the oracle's log_j2 at random
    deformations from random committed states, elastic and far past yield, and at a pure
    stretch with two equal eigenvalues (the degenerate case of the eigenbasis formula)."""
    from oracle import finite

    rng = np.random.default_rng(seed)
    for scale in (2e-4, 3e-2):
        F = np.eye(3) + scale * rng.standard_normal((3, 3))
        if seed == 0:
            F = np.diag([1.0 + scale, 1.0 - scale / 3, 1.0 - scale / 3])
        Hp = 1e-3 * rng.standard_normal((3, 3))
        Hp = 0.5 * (Hp + Hp.T)
        Hp -= np.trace(Hp) / 3 * np.eye(3)
        p = abs(1e-3 * rng.standard_normal())
        G = _G_of_F(F)
        S_o, Hp_o, p_o = finite.log_j2(G[None, :, :, None], (LAM, MU, SIG0), Hp[None, :, :, None],
                                       np.array([[p]]))
        st = [Hp[0, 0], Hp[1, 1], Hp[2, 2], Hp[1, 2], Hp[0, 2], Hp[0, 1], p]
        S, stn = Fm.fftm_host_log_j2(G.reshape(9), (LAM, MU, SIG0), st)
        ref = S_o[0, :, :, 0].reshape(9)
        assert np.abs(S - ref).max() <= 1e-12 * np.abs(ref).max() + 1e-18, (scale, S, ref)
        H1 = Hp_o[0, :, :, 0]
        st_ref = [H1[0, 0], H1[1, 1], H1[2, 2], H1[1, 2], H1[0, 2], H1[0, 1], p_o[0, 0]]
        assert np.abs(stn - st_ref).max() <= 1e-12 * (np.abs(st_ref).max() + 1e-3), (scale, stn, st_ref)


@pytest.mark.parametrize("case", ["periodic", "not_normal_mixed", "faces_differ"])
def test_c0_green_outside_its_conditions_is_refused(case):
    n = (6, 4, 4)
    ph = np.zeros(n, np.uint16)
    bc = [[["D", "N", "N"]] * 2, [["D", "N", "D"]] * 2, [["N", "N", "D"]] * 2]  # normal-mixed
    scheme = "HEX1"
    if case == "periodic":
        bc[2] = [["P"] * 3] * 2
    elif case == "not_normal_mixed":
        bc[1] = [["D"] * 3] * 2
    else:
        bc[0] = [["D", "N", "N"], ["N", "D", "D"]]
    desc, keep = F.make_desc(n, ph, [(ISO_ELASTIC, (LAM, MU), Q1)], bc, scheme=scheme, green="C0",
                             lambda0=LAM, mu0=MU, tol=1e-8, max_iter=100)
    with pytest.raises(F.FFTMError) as e:
        F.fftm_problem_workspace_bytes(desc)
    assert e.value.status == F.FFTM_E_UNSUPPORTED


@pytest.mark.parametrize("scheme", ["HEX1", "TETRA2"])
def test_c0_green_within_its_conditions_is_accepted(scheme):
    n = (6, 4, 4)
    bc = [[["D", "N", "N"]] * 2, [["D", "N", "D"]] * 2, [["N", "N", "D"]] * 2]
    desc, keep = F.make_desc(n, np.zeros(n, np.uint16), [(ISO_ELASTIC, (LAM, MU), Q1)], bc, green="C0",
                             scheme=scheme, lambda0=LAM, mu0=MU, tol=1e-8, max_iter=100)
    assert F.fftm_problem_workspace_bytes(desc) > 0
