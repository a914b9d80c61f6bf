"""Host-side logic of the library, checked against the oracle without a GPU.

* The dense 1D transform matrices the tensor-core path contracts with are the Table 1
  sums (the DFT in halfcomplex order), and the inverse matrices invert them.
* The normal-mixed strain increment the solve loop applies is the oracle's.
* Bad arguments are refused.
"""

import os
import shutil

import numpy as np
import pytest

from oracle import transforms as T
from oracle.mixed import mixed_increment

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")

KINDS = ["DFT", "DCT1", "DCT3", "DST1", "DST3"]


@pytest.fixture(scope="module")
def F():
    from paper_2607_05929_gb300 import build
    from paper_2607_05929_gb300 import fftm

    build.build()
    fftm.load_library()
    return fftm


def _table1(kind, n):
    return T.r2hc_matrix(n) if kind == "DFT" else T.forward_matrix(kind, n).real


@pytest.mark.parametrize("n", [2, 3, 8, 12, 17, 64])
@pytest.mark.parametrize("kind", KINDS)
def test_dense_forward_matrices_are_the_table1_sums(F, kind, n):
    got = F.fftm_host_dense_transform(kind, n)
    ref = _table1(kind, n)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() < 1e-13 * n


@pytest.mark.parametrize("n", [2, 3, 8, 12, 17, 64])
@pytest.mark.parametrize("kind", KINDS)
def test_dense_inverse_matrices_invert_the_forward_ones(F, kind, n):
    fwd = F.fftm_host_dense_transform(kind, n)
    inv = F.fftm_host_dense_transform(kind, n, inverse=True)
    assert np.abs(inv @ fwd - np.eye(fwd.shape[0])).max() < 1e-12 * n
    assert np.abs(inv - np.linalg.inv(_table1(kind, n))).max() < 1e-12 * n


def test_mixed_increment_is_the_oracles(F):
    rng = np.random.default_rng(5)
    for mask in [0b111110, 0b000110, 0b111000, 0b000001, 0b101010, 0b111111]:
        a = rng.standard_normal((3, 3))
        sig = a + a.T
        lam0, mu0 = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
        got = F.fftm_host_mixed_increment(sig, mask, lam0, mu0)
        ref = mixed_increment(sig, mask, lam0, mu0)
        assert np.abs(got - ref).max() < 1e-14 * np.abs(ref).max() + 1e-300


def test_bad_host_arguments_are_refused(F):
    with pytest.raises(F.FFTMError):
        F.fftm_host_dense_transform(7, 8)
    with pytest.raises(F.FFTMError):
        F.fftm_host_dense_transform("DCT1", 1)
    with pytest.raises(F.FFTMError):
        F.fftm_host_mixed_increment(np.eye(3), 1 << 6, 1.0, 1.0)
    with pytest.raises(F.FFTMError):
        F.fftm_host_mixed_increment(np.eye(3), 1, 1.0, 0.0)


def test_dt1d_refuses_bad_arguments_before_any_device_work(F):
    """fftm_dt1d checks its kind, length and arrays before it touches a device."""
    with pytest.raises(F.FFTMError):
        F.fftm_dt1d(7, 8, np.zeros(8))
    with pytest.raises(F.FFTMError):
        F.fftm_dt1d("DCT1", 1, np.zeros(2))
    with pytest.raises(F.FFTMError):
        F.fftm_dt1d("DST1", 5000, np.zeros(4999))


def test_reference_medium_auto_is_half_the_extremes_over_the_phases(F):
    """FFTM_REF_AUTO: (max + min) / 2 of each Lame coefficient over the phases' pairs (isotropic,
    J2: lambda, mu; cubic: C12 and the mid-range shear modulus; Neo-Hooke: K - 2 mu / 3, mu)."""
    q = (1.0, 0.0, 0.0, 0.0)
    mats = [(F.FFTM_LAW_ISO_ELASTIC, (1.0, 2.0), q), (F.FFTM_LAW_CUBIC_ELASTIC, (168.0, 121.0, 75.0), q),
            (F.FFTM_LAW_NEO_HOOKE, (4.0, 10.0), q), (F.FFTM_LAW_J2_LINHARD, (3.0, 0.5, 0.1, 1.0), q)]
    lams = [1.0, 121.0, 10.0 - 8.0 / 3.0, 3.0]
    mus = [2.0, 0.5 * (75.0 + 0.5 * (168.0 - 121.0)), 4.0, 0.5]
    n = (4, 4, 4)
    bc = [[["D"] * 3] * 2, [["P"] * 3] * 2, [["P"] * 3] * 2]
    phase = np.zeros(n, dtype=np.uint16)
    desc, keep = F.make_desc(n, phase, mats, bc, lambda0=F.FFTM_REF_AUTO, mu0=F.FFTM_REF_AUTO)
    l0, m0 = F.fftm_host_reference_medium(desc)
    assert l0 == 0.5 * (max(lams) + min(lams)) and m0 == 0.5 * (max(mus) + min(mus))
    desc, keep = F.make_desc(n, phase, mats, bc, lambda0=7.0, mu0=F.FFTM_REF_AUTO)
    assert F.fftm_host_reference_medium(desc) == (7.0, 0.5 * (max(mus) + min(mus)))
    desc, keep = F.make_desc(n, phase, mats, bc, lambda0=7.0, mu0=3.0)
    assert F.fftm_host_reference_medium(desc) == (7.0, 3.0)
    # the descriptor checks see the resolved values: AUTO is accepted, another negative is not
    desc, keep = F.make_desc(n, phase, mats[:1], bc, lambda0=F.FFTM_REF_AUTO, mu0=F.FFTM_REF_AUTO)
    assert F.fftm_problem_workspace_bytes(desc) > 0
    desc, keep = F.make_desc(n, phase, mats[:1], bc, lambda0=1.0, mu0=-2.0)
    with pytest.raises(F.FFTMError):
        F.fftm_problem_workspace_bytes(desc)
