"""GB300 (sm_103a) hot path of the DTT/FFT displacement-based fixed-point solver.

The compute path is the C-ABI library libfftm.so (include/fftm.h); this
package holds its CUDA sources (csrc/), the in-tree build (build.py) and the
thin ctypes binding (fftm.py).
"""

from . import fftm  # noqa: F401
from .fftm import *  # noqa: F401,F403
