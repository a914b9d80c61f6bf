"""The test export fftm_dt1d: every 1D transform kind of Table 1 and its inverse, computed on the
GPU by the library's FP64 transform pass, against the oracle's dense matrices (the Table 1 sums,
the R2HC DFT) on lengths with odd, even and composite sizes; and the round trip."""

import numpy as np
import pytest

from oracle.transforms import forward_matrix, inverse_matrix, r2hc_matrix
from paper_2607_05929_gb300 import build
from paper_2607_05929_gb300 import fftm as F

pytestmark = pytest.mark.gpu

KINDS = ["DFT", "DCT1", "DCT3", "DST1", "DST3"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    F.load_library()


def _matrices(kind, n):
    if kind == "DFT":
        M = r2hc_matrix(n)
        return M, np.linalg.inv(M)
    return forward_matrix(kind, n), inverse_matrix(kind, n)


@pytest.mark.parametrize("n", [6, 9, 16, 48])
@pytest.mark.parametrize("kind", KINDS)
def test_dt1d_matches_the_oracle(kind, n):
    Mf, Mi = _matrices(kind, n)
    L = Mf.shape[0]
    rng = np.random.default_rng(7 * n + KINDS.index(kind))
    x = rng.standard_normal(L)
    X = F.fftm_dt1d(kind, n, x)
    ref = Mf @ x
    assert np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref)
    back = F.fftm_dt1d(kind, n, X, inverse=True)
    assert np.linalg.norm(back - x) <= 1e-12 * np.linalg.norm(x)
    assert np.linalg.norm(F.fftm_dt1d(kind, n, ref, inverse=True) - Mi @ ref) <= 1e-12 * np.linalg.norm(x)


def test_dt1d_refuses_bad_arguments():
    with pytest.raises(F.FFTMError):
        F.fftm_dt1d(7, 8, np.zeros(8))
    with pytest.raises(F.FFTMError):
        F.fftm_dt1d("DCT1", 1, np.zeros(2))
