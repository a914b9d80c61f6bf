"""fftm_residual_noalloc's binding refuses buffers the residual kernels would overrun (no GPU).

The C entry point reads u and writes D as 3 N1 N2 N3 elements of the problem's precision and
writes 3 doubles of norms; it cannot see the size or type of a device pointer.  The binding
therefore checks every buffer against fftm_problem_layout before the call.  The checks are
host logic, exercised here with stand-ins for CUDA tensors.
"""

import pytest

from paper_2607_05929_gb300 import fftm as F


class _Dev:
    def __init__(self, index):
        self.index = index


class FakeTensor:
    """The attributes of a torch tensor that check_noalloc_args reads."""

    def __init__(self, numel, itemsize, floating=True, cuda=True, contiguous=True, device=0):
        self._n, self._sz, self._fp, self._c = numel, itemsize, floating, contiguous
        self.is_cuda = cuda
        self.device = _Dev(device)
        self.dtype = f"fake{'float' if floating else 'int'}{8 * itemsize}"

    def numel(self):
        return self._n

    def element_size(self):
        return self._sz

    def is_floating_point(self):
        return self._fp

    def is_contiguous(self):
        return self._c


N = (5, 4, 3)
NEED = 3 * 5 * 4 * 3
FP64 = (N, F.FFTM_FP64, 0)
FP32 = (N, F.FFTM_FP32, 0)


def test_matching_buffers_are_accepted():
    F.check_noalloc_args(FP64, FakeTensor(NEED, 8), FakeTensor(NEED, 8), FakeTensor(3, 8))
    F.check_noalloc_args(FP32, FakeTensor(NEED, 4), FakeTensor(NEED, 4), FakeTensor(4, 8))
    F.check_noalloc_args((N, F.FFTM_FP32_TC, 0), FakeTensor(NEED, 4), FakeTensor(NEED, 4), FakeTensor(3, 8))


@pytest.mark.parametrize("layout,u,D,norms,what", [
    (FP64, FakeTensor(NEED, 4), FakeTensor(NEED, 8), FakeTensor(3, 8), "u_dev: dtype"),     # FP32 u, FP64 problem
    (FP32, FakeTensor(NEED, 4), FakeTensor(NEED, 8), FakeTensor(3, 8), "D_dev: dtype"),     # FP64 D, FP32 problem
    (FP64, FakeTensor(NEED, 8), FakeTensor(NEED - 1, 8), FakeTensor(3, 8), "D_dev: "),      # short D
    (FP64, FakeTensor(NEED + 3, 8), FakeTensor(NEED, 8), FakeTensor(3, 8), "u_dev: "),      # long u
    (FP64, FakeTensor(NEED, 8), FakeTensor(NEED, 8), FakeTensor(2, 8), "norms_dev"),        # short norms
    (FP64, FakeTensor(NEED, 8), FakeTensor(NEED, 8), FakeTensor(3, 4), "norms_dev"),        # float32 norms
    (FP64, FakeTensor(NEED, 8), FakeTensor(NEED, 8, floating=False), FakeTensor(3, 8), "D_dev: dtype"),
    (FP64, FakeTensor(NEED, 8, cuda=False), FakeTensor(NEED, 8), FakeTensor(3, 8), "u_dev: a contiguous"),
    (FP64, FakeTensor(NEED, 8), FakeTensor(NEED, 8, contiguous=False), FakeTensor(3, 8), "D_dev: a contiguous"),
    (FP64, FakeTensor(NEED, 8), FakeTensor(NEED, 8), FakeTensor(3, 8, device=1), "norms_dev: on cuda:1"),
])
def test_mismatched_buffers_are_refused(layout, u, D, norms, what):
    with pytest.raises(ValueError, match=what):
        F.check_noalloc_args(layout, u, D, norms)
