"""Marshalling between the oracle's arrays and the C ABI's dense layouts (tests only)."""

import numpy as np

from paper_2607_05929_gb300 import fftm as F
from oracle.bc import dof_range
from oracle.transforms import forward_matrix, r2hc_matrix


def node_to_abi(u):
    """oracle node field (3, N1, N2, N3) [q, x, y, z] -> dense ABI array (3, N3, N2, N1)."""
    return np.ascontiguousarray(np.asarray(u).transpose(0, 3, 2, 1))


def node_from_abi(a):
    return np.asarray(a).transpose(0, 3, 2, 1)


def voxel_from_abi(a, npp, nc, n):
    """dense ABI voxel field -> (npp, nc, n1, n2, n3)."""
    return np.asarray(a).reshape(npp, nc, n[2], n[1], n[0]).transpose(0, 1, 4, 3, 2)


def sym6(P):
    """(npp, 3, 3, ...) -> (npp, 6, ...) in the ABI order 11, 22, 33, 23, 13, 12."""
    return np.stack([P[:, 0, 0], P[:, 1, 1], P[:, 2, 2], P[:, 1, 2], P[:, 0, 2], P[:, 0, 1]], axis=1)


class GpuProblem:
    """A library problem built from a synthetic.Workload (host buffers for all transfers)."""

    def __init__(self, wl, precision="fp64", ctx=None, tol=None, max_iter=None):
        self.wl = wl
        self.dtype = np.float64 if precision == "fp64" else np.float32  # fp32 and fp32_tc
        self.ctx = ctx if ctx is not None else F.fftm_ctx_create(0, None)
        mats = [(m.law, m.params, m.quat) for m in wl.materials]
        desc, self._keep = F.make_desc(
            wl.n, wl.phase, mats, wl.bc, scheme=wl.scheme, green=wl.green, lambda0=wl.lambda0, mu0=wl.mu0,
            precision=precision, tol=wl.tol if tol is None else tol,
            max_iter=wl.max_iter if max_iter is None else max_iter, h=wl.h,
            anderson_depth=wl.anderson_depth, anderson_period=wl.anderson_period)
        self.p = F.fftm_problem_create(self.ctx, desc)
        F.fftm_set_load(self.p, wl.A, wl.b, wl.Q)
        self.N = tuple(wl.n[a] if wl.bc[a][0][0] == "P" else wl.n[a] + 1 for a in range(3))
        self.npp = 2 if wl.scheme == "TETRA2" else 1

    def close(self):
        F.fftm_problem_destroy(self.p)

    def set_node(self, field, u):
        F.fftm_set_field(self.p, field, node_to_abi(u).astype(self.dtype))

    def get_node(self, field):
        out = np.zeros((3, self.N[2], self.N[1], self.N[0]), dtype=self.dtype)
        F.fftm_get_field(self.p, field, out)
        return node_from_abi(out).astype(np.float64)

    def set_load(self, A, b, Q, mixed=0, T=None):
        F.fftm_set_load(self.p, A, b, Q, mixed=mixed, T=T)

    def get_voxel(self, field):
        n = self.wl.n
        nc = F.fftm_field_bytes(self.p, field) // (np.dtype(self.dtype).itemsize * self.npp * n[0] * n[1] * n[2])
        out = np.zeros(self.npp * nc * n[0] * n[1] * n[2], dtype=self.dtype)
        F.fftm_get_field(self.p, field, out)
        return voxel_from_abi(out, self.npp, nc, n).astype(np.float64)


def oracle_r2r_forward(g, kinds, n, N):
    """3D forward DT in the library's storage: DCT/DST coefficient k at node position lo + k,
    periodic axes in halfcomplex order (real definitions: Table 1 sums and the R2HC DFT)."""
    sl = tuple(slice(*dof_range(kinds[a], n[a])) for a in range(3))
    x = np.asarray(g, dtype=np.float64)[sl]
    for a in range(3):
        M = r2hc_matrix(n[a]) if kinds[a] == "DFT" else forward_matrix(kinds[a], n[a])
        x = np.moveaxis(np.moveaxis(x, a, -1) @ M.T, -1, a)
    out = np.zeros(N)
    out[sl] = x
    return out


def rel_l2(a, b):
    nb = np.linalg.norm(np.ravel(b))
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / (nb if nb > 0 else 1.0)
