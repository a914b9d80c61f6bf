"""Thin ctypes binding of include/fftm.h (argument marshalling only).

Every function here forwards to the C function of the same name in
libfftm.so; all arithmetic runs in the library's CUDA kernels.  Device
memory handed to the library comes from PyTorch tensors (``data_ptr``), and
the CUDA stream from ``torch.cuda.current_stream()``.  Importing this module
fails loudly when the library has not been built: there is no fallback.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfftm.so")

# status codes
FFTM_OK = 0
FFTM_NOT_CONVERGED = 1
FFTM_E_INVALID = -1
FFTM_E_NOMEM = -2
FFTM_E_CUDA = -3
FFTM_E_DIVERGED = -4
FFTM_E_UNSUPPORTED = -5
FFTM_E_TIMEOUT = -6
# enums
FFTM_BC_PERIODIC, FFTM_BC_DIRICHLET, FFTM_BC_NEUMANN = 0, 1, 2
FFTM_HEX1, FFTM_TETRA2 = 0, 1
FFTM_GREEN_B0, FFTM_GREEN_MU0, FFTM_GREEN_C0 = 0, 1, 2
FFTM_FP64, FFTM_FP32, FFTM_FP32_TC, FFTM_FP32_TF32 = 0, 1, 2, 3
FFTM_LAW_ISO_ELASTIC, FFTM_LAW_CUBIC_ELASTIC, FFTM_LAW_J2_LINHARD, FFTM_LAW_B0_LINEAR = 0, 1, 2, 3
FFTM_LAW_SVK_CUBIC, FFTM_LAW_NEO_HOOKE, FFTM_LAW_CP_FCC, FFTM_LAW_LOG_J2 = 4, 5, 6, 7
FFTM_FIELD_U, FFTM_FIELD_WORK, FFTM_FIELD_GRAD, FFTM_FIELD_STRESS, FFTM_FIELD_D, FFTM_FIELD_STATE = 0, 1, 2, 3, 4, 5
FFTM_FIELD_U_LO = 6
FFTM_REF_AUTO = -1.0  # fftm_problem_desc.lambda0 / mu0: the reference medium from the phases
FFTM_OPT_RESIDUAL_PASSES, FFTM_OPT_RESIDUAL_TILE, FFTM_OPT_DEVICE_LOOP, FFTM_OPT_CUDA_GRAPH = 0, 1, 2, 3
FFTM_OP_RESIDUAL, FFTM_OP_DT_FORWARD, FFTM_OP_GREEN, FFTM_OP_DT_INVERSE, FFTM_OP_GREEN_UPDATE = 0, 1, 2, 3, 4

# every symbol include/fftm.h declares
EXPORTS = [
    "fftm_last_error", "fftm_version", "fftm_ctx_create", "fftm_ctx_destroy",
    "fftm_problem_workspace_bytes", "fftm_problem_create", "fftm_problem_create_in", "fftm_problem_destroy",
    "fftm_set_phase", "fftm_set_load", "fftm_set_face_traction", "fftm_set_load_field", "fftm_get_load", "fftm_solve_step", "fftm_field_bytes",
    "fftm_get_field", "fftm_set_field", "fftm_problem_layout", "fftm_set_option", "fftm_tuning_table", "fftm_device_fma_rate", "fftm_apply", "fftm_kernel_launches",
    "fftm_reset_state", "fftm_set_profiling", "fftm_kernel_times", "fftm_residual_noalloc",
    "fftm_server_create", "fftm_server_submit", "fftm_server_poll", "fftm_server_pending", "fftm_server_destroy",
    "fftm_server_inject_start_failures", "fftm_server_set_option",
    "fftm_host_dense_transform", "fftm_host_mixed_increment", "fftm_host_log_j2", "fftm_dt1d",
    "fftm_host_reference_medium",
]
FFTM_DT_KINDS = {"DFT": 0, "DCT1": 1, "DCT3": 2, "DST1": 3, "DST3": 4}
FFTM_KCAT_NAMES = ["residual", "pass_x", "pass_y", "pass_z_fused", "anderson", "other"]


class fftm_material(ctypes.Structure):
    _fields_ = [("law", ctypes.c_int), ("params", ctypes.c_double * 12), ("quat", ctypes.c_double * 4)]


class fftm_problem_desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3),
        ("phase", ctypes.POINTER(ctypes.c_uint16)), ("n_phases", ctypes.c_int),
        ("materials", ctypes.POINTER(fftm_material)),
        ("bc", ((ctypes.c_int * 3) * 2) * 3),
        ("scheme", ctypes.c_int), ("green", ctypes.c_int),
        ("lambda0", ctypes.c_double), ("mu0", ctypes.c_double),
        ("precision", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
        ("anderson_depth", ctypes.c_int), ("anderson_period", ctypes.c_int),
    ]


class fftm_load(ctypes.Structure):
    _fields_ = [("A", (ctypes.c_double * 3) * 3), ("b", ctypes.c_double * 3), ("Q", (ctypes.c_double * 6) * 3),
                ("T", ((ctypes.c_double * 3) * 2) * 3), ("mixed", ctypes.c_int)]


class fftm_request(ctypes.Structure):
    _fields_ = [("desc", ctypes.c_void_p), ("loads", ctypes.c_void_p), ("n_loads", ctypes.c_int),
                ("u_out", ctypes.c_void_p), ("u_out_bytes", ctypes.c_size_t)]


class fftm_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("steps", ctypes.c_int),
                ("converged_steps", ctypes.c_int), ("iterations", ctypes.c_int), ("err", ctypes.c_double),
                ("mean_P", ctypes.c_double * 6), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_end", ctypes.c_double), ("message", ctypes.c_char * 160)]


class fftm_step_report(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("err", ctypes.c_double),
        ("n_accelerated", ctypes.c_int), ("mean_P", ctypes.c_double * 6), ("mean_G", ctypes.c_double * 9),
    ]


class FFTMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fftm status {status}: {msg}")
        self.status = status


_lib = None


def load_library(path=LIB_PATH):
    """Load libfftm.so (raises if it is missing: build it with paper_2607_05929_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: the CUDA library must be built (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "fftm_last_error": ([], ctypes.c_char_p),
        "fftm_version": ([], ctypes.c_int),
        "fftm_ctx_create": ([P(vp), ctypes.c_int, vp], ctypes.c_int),
        "fftm_ctx_destroy": ([vp], ctypes.c_int),
        "fftm_problem_workspace_bytes": ([P(fftm_problem_desc), P(ctypes.c_size_t)], ctypes.c_int),
        "fftm_problem_create": ([vp, P(fftm_problem_desc), P(vp)], ctypes.c_int),
        "fftm_problem_create_in": ([vp, P(fftm_problem_desc), vp, ctypes.c_size_t, P(vp)], ctypes.c_int),
        "fftm_problem_destroy": ([vp], ctypes.c_int),
        "fftm_set_phase": ([vp, P(ctypes.c_uint16)], ctypes.c_int),
        "fftm_set_load": ([vp, P(fftm_load)], ctypes.c_int),
        "fftm_get_load": ([vp, P(fftm_load)], ctypes.c_int),
        "fftm_set_face_traction": ([vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, ctypes.c_size_t], ctypes.c_int),
        "fftm_set_load_field": ([vp, vp, ctypes.c_int, ctypes.c_size_t], ctypes.c_int),
        "fftm_host_dense_transform": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_double),
                                       P(ctypes.c_int)], ctypes.c_int),
        "fftm_dt1d": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_double),
                       P(ctypes.c_double)], ctypes.c_int),
        "fftm_host_reference_medium": ([P(fftm_problem_desc), P(ctypes.c_double), P(ctypes.c_double)],
                                       ctypes.c_int),
        "fftm_host_mixed_increment": ([P(ctypes.c_double), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       P(ctypes.c_double)], ctypes.c_int),
        "fftm_host_log_j2": ([P(ctypes.c_double)] * 5, ctypes.c_int),
        "fftm_solve_step": ([vp, P(fftm_step_report), P(ctypes.c_double), P(ctypes.c_int), ctypes.c_int],
                            ctypes.c_int),
        "fftm_field_bytes": ([vp, ctypes.c_int, P(ctypes.c_size_t)], ctypes.c_int),
        "fftm_problem_layout": ([vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)], ctypes.c_int),
        "fftm_set_option": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "fftm_device_fma_rate": ([ctypes.c_int, ctypes.c_int, P(ctypes.c_double)], ctypes.c_int),
        "fftm_tuning_table": ([ctypes.c_char_p, ctypes.c_size_t, P(ctypes.c_size_t)], ctypes.c_int),
        "fftm_get_field": ([vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_size_t], ctypes.c_int),
        "fftm_set_field": ([vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_size_t], ctypes.c_int),
        "fftm_apply": ([vp, ctypes.c_int, P(ctypes.c_double)], ctypes.c_int),
        "fftm_kernel_launches": ([vp, P(ctypes.c_longlong)], ctypes.c_int),
        "fftm_reset_state": ([vp], ctypes.c_int),
        "fftm_set_profiling": ([vp, ctypes.c_int], ctypes.c_int),
        "fftm_kernel_times": ([vp, P(ctypes.c_double), P(ctypes.c_longlong), ctypes.c_int], ctypes.c_int),
        "fftm_residual_noalloc": ([vp, vp, vp, vp], ctypes.c_int),
        "fftm_server_create": ([ctypes.c_int, ctypes.c_size_t, ctypes.c_int, P(vp)], ctypes.c_int),
        "fftm_server_submit": ([vp, P(fftm_request), P(ctypes.c_longlong)], ctypes.c_int),
        "fftm_server_poll": ([vp, P(fftm_result), ctypes.c_int, ctypes.c_int, P(ctypes.c_int)], ctypes.c_int),
        "fftm_server_pending": ([vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_size_t)], ctypes.c_int),
        "fftm_server_destroy": ([vp], ctypes.c_int),
        "fftm_server_inject_start_failures": ([ctypes.c_int], ctypes.c_int),
        "fftm_server_set_option": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status):
    if status < 0:
        raise FFTMError(status, load_library().fftm_last_error().decode())
    return status


# ---------------------------------------------------------------------------------------
def fftm_last_error():
    return load_library().fftm_last_error().decode()


def fftm_version():
    return load_library().fftm_version()


def fftm_ctx_create(device=0, stream=None):
    """stream: a cudaStream_t as int, a torch.cuda.Stream, or None (legacy default stream)."""
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    ctx = ctypes.c_void_p()
    _check(load_library().fftm_ctx_create(ctypes.byref(ctx), int(device), ctypes.c_void_p(stream or 0)))
    return ctx


def fftm_ctx_destroy(ctx):
    return _check(load_library().fftm_ctx_destroy(ctx))


def make_desc(n, phase, materials, bc, scheme="HEX1", green="B0", lambda0=0.0, mu0=1.0, precision="fp64",
              tol=1e-6, max_iter=1000, h=(1.0, 1.0, 1.0), anderson_depth=4, anderson_period=3):
    """Marshal a problem description.

    phase: integer array indexed [x, y, z]; materials: list of (law, params, quat);
    bc[a][f][q] in {'P','D','N'}.  Returns (desc, keepalive) -- keep `keepalive`
    alive until fftm_problem_create returns.
    """
    ph = np.ascontiguousarray(np.asarray(phase, dtype=np.uint16).transpose(2, 1, 0))  # x fastest
    mats = (fftm_material * len(materials))()
    for i, (law, params, quat) in enumerate(materials):
        mats[i].law = int(law)
        for k, v in enumerate(params):
            mats[i].params[k] = float(v)
        for k, v in enumerate(quat):
            mats[i].quat[k] = float(v)
    d = fftm_problem_desc()
    for a in range(3):
        d.n[a] = int(n[a])
        d.h[a] = float(h[a])
    d.phase = ph.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16))
    d.n_phases = len(materials)
    d.materials = ctypes.cast(mats, ctypes.POINTER(fftm_material))
    code = {"P": FFTM_BC_PERIODIC, "D": FFTM_BC_DIRICHLET, "N": FFTM_BC_NEUMANN}
    for a in range(3):
        for f in range(2):
            for q in range(3):
                d.bc[a][f][q] = code[bc[a][f][q]]
    d.scheme = FFTM_TETRA2 if scheme == "TETRA2" else FFTM_HEX1
    d.green = {"B0": FFTM_GREEN_B0, "MU0": FFTM_GREEN_MU0, "C0": FFTM_GREEN_C0}[green]
    d.lambda0 = float(lambda0)
    d.mu0 = float(mu0)
    d.precision = {"fp64": FFTM_FP64, "fp32": FFTM_FP32, "float32": FFTM_FP32,
                   "fp32_tc": FFTM_FP32_TC, "fp32_tf32": FFTM_FP32_TF32}[precision]
    d.tol = float(tol)
    d.max_iter = int(max_iter)
    d.anderson_depth = int(anderson_depth)
    d.anderson_period = int(anderson_period)
    return d, (ph, mats)


def fftm_problem_workspace_bytes(desc):
    b = ctypes.c_size_t()
    _check(load_library().fftm_problem_workspace_bytes(ctypes.byref(desc), ctypes.byref(b)))
    return b.value


def fftm_problem_create_in(ctx, desc, workspace):
    """fftm_problem_create inside a caller's device buffer (a contiguous CUDA tensor; keep it alive
    until fftm_problem_destroy)."""
    ptr, dev, nb = _ptr_of(workspace)
    if not dev:
        raise ValueError("the workspace must be device memory")
    p = ctypes.c_void_p()
    _check(load_library().fftm_problem_create_in(ctx, ctypes.byref(desc), ctypes.c_void_p(ptr), nb, ctypes.byref(p)))
    return p


def fftm_problem_create(ctx, desc):
    p = ctypes.c_void_p()
    _check(load_library().fftm_problem_create(ctx, ctypes.byref(desc), ctypes.byref(p)))
    return p


def fftm_problem_destroy(p):
    return _check(load_library().fftm_problem_destroy(p))


def fftm_set_phase(p, phase):
    ph = np.ascontiguousarray(np.asarray(phase, dtype=np.uint16).transpose(2, 1, 0))
    return _check(load_library().fftm_set_phase(p, ph.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16))))


def fftm_set_phase_raw(p, host_ptr):
    """fftm_set_phase with a host pointer to an x-fastest uint16 map (e.g. pinned memory)."""
    return _check(load_library().fftm_set_phase(p, ctypes.cast(ctypes.c_void_p(int(host_ptr)),
                                                                ctypes.POINTER(ctypes.c_uint16))))


def fftm_set_load(p, A, b=(0.0, 0.0, 0.0), Q=None, mixed=0, T=None):
    """u*_q = A[q] . x + b[q] + sum_k Q[q][k] m_k(x), m = (x1^2, x2^2, x3^2, x2 x3, x1 x3, x1 x2);
    mixed: normal-mixed mask (Voigt order 11, 22, 33, 23, 13, 12) of the strain components
    adjusted so that the mean stress vanishes in them; T[axis][face][component]: uniform
    tractions on Neumann faces."""
    ld = fftm_load()
    for q in range(3):
        for a in range(3):
            ld.A[q][a] = float(A[q][a])
        ld.b[q] = float(b[q])
        for k in range(6):
            ld.Q[q][k] = 0.0 if Q is None else float(Q[q][k])
    if T is not None:
        for a in range(3):
            for f in range(2):
                for q in range(3):
                    ld.T[a][f][q] = float(T[a][f][q])
    ld.mixed = int(mixed)
    return _check(load_library().fftm_set_load(p, ctypes.byref(ld)))


def fftm_dt1d(kind, n, x, inverse=False, device=0):
    """The 1D transform of Table 1 (or its inverse) of the L values x, on the GPU by the
    library's FP64 transform pass; returns the L outputs."""
    k = FFTM_DT_KINDS[kind] if isinstance(kind, str) else int(kind)
    xin = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(xin)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load_library().fftm_dt1d(int(device), k, int(n), int(bool(inverse)), xin.ctypes.data_as(dp),
                                    out.ctypes.data_as(dp)))
    return out


def fftm_host_reference_medium(desc):
    """(lambda0, mu0) a descriptor asks for, FFTM_REF_AUTO resolved from its phases (host only)."""
    l0, m0 = ctypes.c_double(), ctypes.c_double()
    _check(load_library().fftm_host_reference_medium(ctypes.byref(desc), ctypes.byref(l0), ctypes.byref(m0)))
    return l0.value, m0.value


def fftm_host_dense_transform(kind, n, inverse=False):
    """The L x L matrix the tensor-core path uses for a 1D transform of Table 1 (host only)."""
    k = FFTM_DT_KINDS[kind] if isinstance(kind, str) else int(kind)
    L = ctypes.c_int(0)
    _check(load_library().fftm_host_dense_transform(k, int(n), int(bool(inverse)), None, ctypes.byref(L)))
    out = np.zeros(L.value * L.value)
    _check(load_library().fftm_host_dense_transform(k, int(n), int(bool(inverse)),
                                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                    ctypes.byref(L)))
    return out.reshape(L.value, L.value)


def fftm_host_log_j2(G, params, st):
    """The library's logarithmic J2 law at one point (host only): G (9,), params (3,), st (7,)
    -> (S (9,), returned state (7,))."""
    dp = ctypes.POINTER(ctypes.c_double)
    g = np.ascontiguousarray(np.asarray(G, dtype=np.float64).reshape(9))
    c = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(3))
    z = np.ascontiguousarray(np.asarray(st, dtype=np.float64).reshape(7))
    S, zn = np.zeros(9), np.zeros(7)
    _check(load_library().fftm_host_log_j2(g.ctypes.data_as(dp), c.ctypes.data_as(dp), z.ctypes.data_as(dp),
                                           S.ctypes.data_as(dp), zn.ctypes.data_as(dp)))
    return S, zn


def fftm_host_mixed_increment(sig, mask, lambda0, mu0):
    """The normal-mixed strain increment for a mean stress (host only)."""
    s = np.ascontiguousarray(np.asarray(sig, dtype=np.float64).reshape(9))
    d = np.zeros(9)
    _check(load_library().fftm_host_mixed_increment(s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(mask),
                                                    float(lambda0), float(mu0),
                                                    d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return d.reshape(3, 3)


def fftm_get_load(p):
    """The current load as (A 3x3, b, Q, mixed), A with the adjusted free components."""
    ld = fftm_load()
    _check(load_library().fftm_get_load(p, ctypes.byref(ld)))
    A = np.array([[ld.A[q][a] for a in range(3)] for q in range(3)])
    return A, np.array(list(ld.b)), np.array([[ld.Q[q][k] for k in range(6)] for q in range(3)]), ld.mixed


def fftm_solve_step(p, history_len=0):
    """Returns (status, report dict, err history array, accel history array)."""
    rep = fftm_step_report()
    eh = np.zeros(max(history_len, 1), dtype=np.float64)
    ah = np.zeros(max(history_len, 1), dtype=np.int32)
    st = _check(load_library().fftm_solve_step(
        p, ctypes.byref(rep), eh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        ah.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(history_len)))
    r = {"iterations": rep.iterations, "converged": bool(rep.converged), "err": rep.err,
         "n_accelerated": rep.n_accelerated, "mean_P": np.array(rep.mean_P[:]),
         "mean_G": np.array(rep.mean_G[:])}
    n = min(history_len, rep.iterations + 1)
    return st, r, eh[:n], ah[:n]


def fftm_field_bytes(p, field):
    b = ctypes.c_size_t()
    _check(load_library().fftm_field_bytes(p, int(field), ctypes.byref(b)))
    return b.value


def fftm_problem_layout(p):
    """(N (3 node dims), precision enum, CUDA device) of a problem."""
    N = (ctypes.c_int * 3)()
    prec, dev = ctypes.c_int(), ctypes.c_int()
    _check(load_library().fftm_problem_layout(p, N, ctypes.byref(prec), ctypes.byref(dev)))
    return tuple(N[:]), prec.value, dev.value


def fftm_set_option(p, option, value):
    return _check(load_library().fftm_set_option(p, int(option), int(value)))


def fftm_device_fma_rate(device=0, fp64=True):
    """Measured FMA throughput of the device in FLOP/s (FP64 or FP32)."""
    r = ctypes.c_double()
    _check(load_library().fftm_device_fma_rate(int(device), int(bool(fp64)), ctypes.byref(r)))
    return r.value


def fftm_tuning_table():
    """The launch-shape choices measured in this process, as text."""
    need = ctypes.c_size_t()
    _check(load_library().fftm_tuning_table(None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check(load_library().fftm_tuning_table(buf, need.value, None))
    return buf.value.decode()


def _ptr_of(buf):
    """(pointer, is_device, nbytes) of a torch tensor or a numpy array."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffer must be C-contiguous")
        return buf.ctypes.data, 0, buf.nbytes
    if not buf.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return buf.data_ptr(), int(buf.is_cuda), buf.numel() * buf.element_size()


def fftm_set_face_traction(p, axis, face, t):
    """Non-uniform tractions on one face: t (numpy array or torch tensor, the problem's precision)
    of shape (3, n_c, n_b) in the ABI order, or None to remove the field."""
    if t is None:
        return _check(load_library().fftm_set_face_traction(p, int(axis), int(face), None, 0, 0))
    ptr, dev, nb = _ptr_of(t)
    return _check(load_library().fftm_set_face_traction(p, int(axis), int(face), ctypes.c_void_p(ptr), dev, nb))


def fftm_set_load_field(p, ustar):
    """u* as a node field (numpy array or torch tensor of the problem's precision, the dense
    layout (3, N3, N2, N1)), or None to remove it."""
    if ustar is None:
        return _check(load_library().fftm_set_load_field(p, None, 0, 0))
    ptr, dev, nb = _ptr_of(ustar)
    return _check(load_library().fftm_set_load_field(p, ctypes.c_void_p(ptr), dev, nb))


def fftm_get_field(p, field, out):
    ptr, dev, nb = _ptr_of(out)
    return _check(load_library().fftm_get_field(p, int(field), ctypes.c_void_p(ptr), dev, nb))


def fftm_set_field(p, field, src):
    ptr, dev, nb = _ptr_of(src)
    return _check(load_library().fftm_set_field(p, int(field), ctypes.c_void_p(ptr), dev, nb))


def fftm_apply(p, op):
    """Returns (status, norms[3])."""
    norms = (ctypes.c_double * 3)()
    st = _check(load_library().fftm_apply(p, int(op), norms))
    return st, np.array(norms[:])


def fftm_kernel_launches(p):
    c = ctypes.c_longlong()
    _check(load_library().fftm_kernel_launches(p, ctypes.byref(c)))
    return c.value


def fftm_reset_state(p):
    return _check(load_library().fftm_reset_state(p))


def fftm_set_profiling(p, enable=True):
    return _check(load_library().fftm_set_profiling(p, int(bool(enable))))


def fftm_kernel_times(p):
    """dict category -> (total ms, launches)."""
    n = len(FFTM_KCAT_NAMES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    _check(load_library().fftm_kernel_times(p, ms, cnt, n))
    return {FFTM_KCAT_NAMES[i]: (ms[i], cnt[i]) for i in range(n)}


def check_noalloc_args(layout, u_dev, D_dev, norms_dev):
    """Refuse buffers the residual kernels would read or write out of bounds: u and D must be
    contiguous CUDA tensors on the problem's device, of the problem's precision (float64 for
    FFTM_FP64, float32 otherwise), with exactly 3 N1 N2 N3 elements; norms a contiguous
    float64 CUDA tensor of at least 3 elements on the same device.  Raises ValueError."""
    N, prec, dev = layout
    want_size = 8 if prec == FFTM_FP64 else 4
    need = 3 * N[0] * N[1] * N[2]
    for name, t in (("u_dev", u_dev), ("D_dev", D_dev), ("norms_dev", norms_dev)):
        if not getattr(t, "is_cuda", False) or not t.is_contiguous():
            raise ValueError(f"{name}: a contiguous CUDA tensor is expected")
        if t.device.index != dev:
            raise ValueError(f"{name}: on cuda:{t.device.index}, the problem is on cuda:{dev}")
    for name, t in (("u_dev", u_dev), ("D_dev", D_dev)):
        if not t.is_floating_point() or t.element_size() != want_size:
            raise ValueError(f"{name}: dtype {t.dtype} does not match the problem precision "
                             f"({'float64' if want_size == 8 else 'float32'})")
        if t.numel() != need:
            raise ValueError(f"{name}: {t.numel()} elements, the node field has 3 x {N} = {need}")
    if not norms_dev.is_floating_point() or norms_dev.element_size() != 8 or norms_dev.numel() < 3:
        raise ValueError("norms_dev: a float64 tensor of at least 3 elements is expected")


def fftm_residual_noalloc(p, u_dev, D_dev, norms_dev):
    """Residual D and norms of a caller-supplied u^f into caller device buffers (torch CUDA
    tensors: u and D in the dense node layout, norms 3 float64); allocates no device memory.
    The buffers are checked against the problem's layout first (check_noalloc_args)."""
    check_noalloc_args(fftm_problem_layout(p), u_dev, D_dev, norms_dev)
    return _check(load_library().fftm_residual_noalloc(p, ctypes.c_void_p(u_dev.data_ptr()),
                                                        ctypes.c_void_p(D_dev.data_ptr()),
                                                        ctypes.c_void_p(norms_dev.data_ptr())))


# ---- serving runtime (include/fftm_server.h) ------------------------------------------
def fftm_server_create(device=0, memory_budget=0, max_slots=4):
    s = ctypes.c_void_p()
    _check(load_library().fftm_server_create(int(device), int(memory_budget), int(max_slots), ctypes.byref(s)))
    return s


def make_loads(loads):
    """[(A, b, Q), ...] -> ctypes array of fftm_load."""
    arr = (fftm_load * len(loads))()
    for k, (A, b, Q) in enumerate(loads):
        for q in range(3):
            for a in range(3):
                arr[k].A[q][a] = float(A[q][a])
            arr[k].b[q] = float(b[q])
            for m in range(6):
                arr[k].Q[q][m] = 0.0 if Q is None else float(Q[q][m])
    return arr


def fftm_server_submit(s, desc, loads, u_out=None):
    """desc: a fftm_problem_desc (from make_desc; its keepalive must live until this returns);
    loads: [(A, b, Q), ...]; u_out: optional C-contiguous numpy array for the final u^f, kept
    alive by the caller until the result is polled.  Returns the request id."""
    la = make_loads(loads)
    req = fftm_request()
    req.desc = ctypes.cast(ctypes.pointer(desc), ctypes.c_void_p)
    req.loads = ctypes.cast(la, ctypes.c_void_p)
    req.n_loads = len(loads)
    if u_out is not None:
        if not u_out.flags["C_CONTIGUOUS"]:
            raise ValueError("u_out must be C-contiguous")
        req.u_out = u_out.ctypes.data
        req.u_out_bytes = u_out.nbytes
    rid = ctypes.c_longlong()
    _check(load_library().fftm_server_submit(s, ctypes.byref(req), ctypes.byref(rid)))
    return rid.value


def fftm_server_poll(s, max_results=64, wait=True):
    """Finished results as dicts (completion order)."""
    out = (fftm_result * max_results)()
    n = ctypes.c_int()
    _check(load_library().fftm_server_poll(s, out, int(max_results), int(bool(wait)), ctypes.byref(n)))
    res = []
    for r in out[:n.value]:
        res.append({"id": r.id, "status": r.status, "steps": r.steps, "converged_steps": r.converged_steps,
                    "iterations": r.iterations, "err": r.err, "mean_P": np.array(r.mean_P[:]),
                    "t_submit": r.t_submit, "t_start": r.t_start, "t_end": r.t_end,
                    "message": r.message.decode(errors="replace")})
    return res


def fftm_server_pending(s):
    q, a, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    _check(load_library().fftm_server_pending(s, ctypes.byref(q), ctypes.byref(a), ctypes.byref(b)))
    return q.value, a.value, b.value


def fftm_server_destroy(s):
    return _check(load_library().fftm_server_destroy(s))


def fftm_server_set_option(srv, option, value):
    return _check(load_library().fftm_server_set_option(srv, int(option), int(value)))


def fftm_server_inject_start_failures(count):
    return _check(load_library().fftm_server_inject_start_failures(int(count)))
