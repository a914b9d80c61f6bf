"""The C-ABI library builds for sm_103a, loads, and exports every symbol the headers in include/ declare.

No compute call is made here (no GPU needed).
"""

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fftm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_2607_05929_gb300 import build, fftm

    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert declared, "no declarations parsed"
    assert sorted(fftm.EXPORTS) == declared
    for name in declared:
        assert hasattr(lib, name), name
    assert fftm.fftm_version() >= 1


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2607_05929_gb300 import fftm

    saved = fftm._lib
    try:
        fftm._lib = None
        with pytest.raises(RuntimeError):
            fftm.load_library(str(tmp_path / "missing.so"))
    finally:
        fftm._lib = saved
