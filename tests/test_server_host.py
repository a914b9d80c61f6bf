"""Serving runtime start-up failures, injected on the host (no GPU, no device fault).

A worker that cannot create its CUDA stream or library context must not leave the server
looking healthy: when no worker starts, fftm_server_create reports FFTM_E_CUDA and returns
no server (so nothing can be queued that no thread would ever run, and no poll can wait
forever).  The failure is injected with the library's host-side hook, which makes the
chosen workers fail before any CUDA call.
"""

import os
import shutil

import pytest

from paper_2607_05929_gb300 import fftm as F

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2607_05929_gb300 import build

    build.build()
    F.load_library()


@pytest.mark.parametrize("slots", [1, 3])
def test_create_fails_when_no_worker_starts(slots):
    F.fftm_server_inject_start_failures(slots)
    try:
        with pytest.raises(F.FFTMError) as e:
            F.fftm_server_create(0, 1 << 30, slots)
        assert e.value.status == F.FFTM_E_CUDA
    finally:
        F.fftm_server_inject_start_failures(0)


def test_injection_hook_rejects_a_negative_count():
    with pytest.raises(F.FFTMError) as e:
        F.fftm_server_inject_start_failures(-1)
    assert e.value.status == F.FFTM_E_INVALID
