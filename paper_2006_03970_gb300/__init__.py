"""GB300-native SsNAL-EN: Python binding of libssnal_en (include/ssnal_en.h).

This module only marshals arguments for the C ABI: every step of the solver
runs in the library's CUDA kernels.  PyTorch provides device memory and the
current CUDA stream.  The functions carry the names of the C entry points
(``ssnal_en_create``, ``ssnal_en_solve``, ``ssnal_en_path`` ...); ``Context``
wraps them for convenience.

There is no CPU fallback: if the shared library is missing or CUDA is not
available the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "F64", "F32", "BF16", "I8_GENO", "I2_GENO", "pack_codes_2bit", "OK", "EINVAL", "ENOMEM", "ENOCONV", "ECUDA", "ETIMEOUT", "ENOTSUP",
    "SsnalError", "Matrix", "Options", "Result", "load_library", "device_matrix", "default_options",
    "ssnal_en_default_options", "ssnal_en_create", "ssnal_en_destroy", "ssnal_en_set_options", "ssnal_en_solve",
    "ssnal_en_solve_batch", "ssnal_en_solve_shared", "ssnal_en_solve_batch_resident", "BatchFit", "ssnal_en_server_set_group", "Instance", "Server", "ssnal_en_server_create", "ssnal_en_server_submit",
    "ssnal_en_server_poll", "ssnal_en_server_destroy", "ssnal_en_server_submit_scaled", "ssnal_en_tune",
    "TunePoint", "ssnal_en_path", "ssnal_en_path_host", "ssnal_en_op_at_y", "ssnal_en_op_at_d", "ssnal_en_op_prox_active",
    "ssnal_en_op_grad",
    "ssnal_en_op_newton", "ssnal_en_profile", "ssnal_en_profile_phases", "ssnal_en_prox_active_static",
    "STATIC_MAX_N", "Context",
]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libssnal_en.so")

F64, F32, BF16, I8_GENO, I2_GENO = 0, 1, 2, 3, 4
OK, EINVAL, ENOMEM, ENOCONV, ECUDA, ETIMEOUT, ENOTSUP = range(7)
_ELEM = {F64: 8, F32: 4, BF16: 2, I8_GENO: 1}
STATIC_MAX_N = 2097152  # SSNAL_EN_STATIC_MAX_N


class SsnalError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {_lib_status(status)} (status {status})")


class Matrix(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("lda", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("data", ctypes.c_void_p), ("col_mean", ctypes.c_void_p),
                ("col_scale", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("sigma0", ctypes.c_double), ("sigma_growth", ctypes.c_double), ("sigma_max", ctypes.c_double),
                ("mu", ctypes.c_double), ("beta", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_al", ctypes.c_int32), ("max_newton", ctypes.c_int32), ("max_ls", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("refine_steps", ctypes.c_int32), ("use_y0", ctypes.c_int32),
                ("ls_fused", ctypes.c_int32), ("syrk_tc", ctypes.c_int32), ("max_active", ctypes.c_int64),
                ("newton_fp64", ctypes.c_int32), ("cg_maxit", ctypes.c_int32), ("cg_above", ctypes.c_int64),
                ("cg_rtol", ctypes.c_double)]


class Instance(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("b", ctypes.c_void_p), ("lambda1", ctypes.c_double),
                ("lambda2", ctypes.c_double), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p)]


class BatchFit(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("b", ctypes.c_void_p), ("lambda1", ctypes.c_double), ("lambda2", ctypes.c_double),
                ("x", ctypes.c_void_p)]


class TunePoint(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("rss", ctypes.c_double), ("gcv", ctypes.c_double),
                ("ebic", ctypes.c_double), ("active", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("al_iters", ctypes.c_int32), ("newton_iters", ctypes.c_int32),
                ("ls_trials", ctypes.c_int32), ("active", ctypes.c_int64), ("kkt1", ctypes.c_double),
                ("kkt3", ctypes.c_double), ("primal_obj", ctypes.c_double), ("dual_gap", ctypes.c_double),
                ("seconds", ctypes.c_double), ("sigma", ctypes.c_double), ("lambda1", ctypes.c_double),
                ("lambda2", ctypes.c_double), ("newton_fp64", ctypes.c_int32), ("cg_iters", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
EXPORTS = ["ssnal_en_default_options", "ssnal_en_status_string", "ssnal_en_create", "ssnal_en_destroy",
           "ssnal_en_set_options", "ssnal_en_solve", "ssnal_en_path", "ssnal_en_path_host", "ssnal_en_op_at_y",
           "ssnal_en_op_at_d", "ssnal_en_solve_batch", "ssnal_en_server_create", "ssnal_en_server_submit",
           "ssnal_en_server_submit_scaled", "ssnal_en_server_poll", "ssnal_en_server_destroy", "ssnal_en_tune",
           "ssnal_en_op_prox_active", "ssnal_en_op_grad", "ssnal_en_op_newton", "ssnal_en_profile",
           "ssnal_en_prox_active_static", "ssnal_en_profile_phases", "ssnal_en_solve_shared",
           "ssnal_en_server_set_group", "ssnal_en_solve_batch_resident"]


def load_library(path: str | None = None):
    """Loads libssnal_en.so (built by paper_2006_03970_gb300.build) and declares the signatures."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(p)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.ssnal_en_default_options.argtypes = [ctypes.POINTER(Options)]
    L.ssnal_en_default_options.restype = None
    L.ssnal_en_status_string.argtypes = [i32]
    L.ssnal_en_status_string.restype = ctypes.c_char_p
    L.ssnal_en_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Matrix), ctypes.POINTER(Options), vp]
    L.ssnal_en_destroy.argtypes = [vp]
    L.ssnal_en_destroy.restype = None
    L.ssnal_en_set_options.argtypes = [vp, ctypes.POINTER(Options)]
    L.ssnal_en_solve.argtypes = [vp, vp, dbl, dbl, vp, vp, ctypes.POINTER(Result)]
    L.ssnal_en_solve_batch.argtypes = [ctypes.POINTER(Instance), ctypes.c_int64, i32, ctypes.POINTER(Result),
                                       ctypes.POINTER(i32)]
    L.ssnal_en_solve_shared.argtypes = [ctypes.POINTER(Instance), i32, ctypes.POINTER(Result), ctypes.POINTER(i32)]
    L.ssnal_en_server_set_group.argtypes = [vp, i32]
    L.ssnal_en_solve_batch_resident.argtypes = [ctypes.POINTER(BatchFit), ctypes.c_int64, ctypes.POINTER(Options),
                                                ctypes.POINTER(Result), ctypes.POINTER(i32), vp]
    L.ssnal_en_server_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Matrix), i32, ctypes.POINTER(Options), i32,
                                         ctypes.c_int64]
    L.ssnal_en_server_submit.argtypes = [vp, i32, ctypes.POINTER(dbl), dbl, dbl, ctypes.POINTER(ctypes.c_int64)]
    L.ssnal_en_server_submit_scaled.argtypes = [vp, i32, ctypes.POINTER(dbl), dbl, dbl,
                                                ctypes.POINTER(ctypes.c_int64)]
    L.ssnal_en_server_poll.argtypes = [vp, ctypes.c_int64, i32, ctypes.POINTER(dbl), ctypes.POINTER(Result),
                                       ctypes.POINTER(dbl), ctypes.POINTER(i32)]
    L.ssnal_en_server_destroy.argtypes = [vp]
    L.ssnal_en_tune.argtypes = [vp, vp, dbl, ctypes.POINTER(dbl), i32, vp, ctypes.POINTER(Result),
                                ctypes.POINTER(TunePoint), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                ctypes.POINTER(i32)]
    L.ssnal_en_server_destroy.restype = None
    L.ssnal_en_path.argtypes = [vp, vp, dbl, ctypes.POINTER(dbl), i32, vp, ctypes.POINTER(Result),
                                ctypes.POINTER(i32)]
    L.ssnal_en_path_host.argtypes = [vp, ctypes.POINTER(dbl), dbl, ctypes.POINTER(dbl), i32, vp,
                                     ctypes.POINTER(Result), ctypes.POINTER(i32)]
    L.ssnal_en_op_at_y.argtypes = [vp, vp, vp]
    L.ssnal_en_op_at_d.argtypes = [vp, vp, vp]
    L.ssnal_en_op_prox_active.argtypes = [vp, vp, vp, dbl, dbl, dbl, vp, vp, ctypes.POINTER(i64)]
    L.ssnal_en_op_grad.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    L.ssnal_en_op_newton.argtypes = [vp, i64, dbl, vp, vp]
    L.ssnal_en_profile_phases.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64)]
    L.ssnal_en_prox_active_static.argtypes = [vp, vp, i64, dbl, dbl, dbl, vp, vp, ctypes.POINTER(i64), vp]
    L.ssnal_en_profile.argtypes = [vp, i32, i32, ctypes.POINTER(dbl), ctypes.POINTER(i64), ctypes.POINTER(dbl),
                                   ctypes.POINTER(i64)]
    for name in EXPORTS:
        if getattr(L, name).restype is ctypes.c_int:
            getattr(L, name).restype = i32
    if path is None:
        _LIB = L
    return L


def _lib_status(status):
    try:
        return load_library().ssnal_en_status_string(int(status)).decode()
    except OSError:
        return "unknown"


def _check(status, where, allow=(OK,)):
    if status not in allow:
        raise SsnalError(status, where)
    return status


def _ptr(t):
    """Device (or host) address of a torch tensor, None for None."""
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def ssnal_en_default_options(**overrides) -> Options:
    o = Options()
    load_library().ssnal_en_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


default_options = ssnal_en_default_options


def pack_codes_2bit(codes: np.ndarray) -> np.ndarray:
    """Packs genotype codes 0..3 of a feature-major (n, m) array four per byte in the
    SSNAL_EN_I2_GENO layout: returns (n, lda / 4) uint8 with lda = m rounded up to 64,
    row i of column j in bits 2 (i mod 4), 2 (i mod 4) + 1 of byte i / 4 of that column
    (rows past m hold code 0)."""
    c = np.asarray(codes)
    n, m = c.shape
    if c.size and (c.min() < 0 or c.max() > 3):
        raise ValueError("2-bit codes must lie in 0..3")
    lda = (m + 63) // 64 * 64
    full = np.zeros((n, lda), dtype=np.uint8)
    full[:, :m] = c
    q = full.reshape(n, lda // 4, 4)
    return (q[:, :, 0] | (q[:, :, 1] << 2) | (q[:, :, 2] << 4) | (q[:, :, 3] << 6)).astype(np.uint8)


def device_matrix(At: np.ndarray, dtype: int = F64, device="cuda"):
    """Copies a feature-major (n, m) array (== column-major A) to the device with a
    16-byte-aligned leading dimension; returns (tensor of shape (n, lda), m).  For
    I2_GENO, At holds the codes 0..3 and the tensor the packed bytes (n, lda / 4)."""
    import torch
    n, m = At.shape
    if dtype == I2_GENO:
        return torch.from_numpy(pack_codes_2bit(At)).to(device), m
    es = _ELEM[dtype]
    q = 16 // es
    lda = (m + q - 1) // q * q
    if dtype == F64:
        host = np.zeros((n, lda), dtype=np.float64)
        host[:, :m] = At
        t = torch.from_numpy(host).to(device)
    elif dtype == F32:
        host = np.zeros((n, lda), dtype=np.float32)
        host[:, :m] = At
        t = torch.from_numpy(host).to(device)
    elif dtype == BF16:
        host = np.zeros((n, lda), dtype=np.uint16)
        host[:, :m] = At  # bf16 bit patterns
        t = torch.from_numpy(host.view(np.int16)).to(device)
    else:
        host = np.zeros((n, lda), dtype=np.int8)
        host[:, :m] = At
        t = torch.from_numpy(host).to(device)
    return t, m


def ssnal_en_create(A, m: int, dtype: int = F64, options: Options | None = None, stream=None,
                    col_mean=None, col_scale=None):
    """A: device tensor (n, lda) holding column-major A ((n, lda / 4) packed bytes for
    I2_GENO).  Returns an opaque context handle."""
    lda = A.shape[1] * 4 if dtype == I2_GENO else A.shape[1]
    mat = Matrix(m=m, n=A.shape[0], lda=lda, dtype=dtype, reserved=0, data=A.data_ptr(),
                 col_mean=col_mean.data_ptr() if col_mean is not None else None,
                 col_scale=col_scale.data_ptr() if col_scale is not None else None)
    ctx = ctypes.c_void_p()
    st = load_library().ssnal_en_create(ctypes.byref(ctx), ctypes.byref(mat),
                                        ctypes.byref(options) if options is not None else None,
                                        _stream_handle(stream))
    _check(st, "ssnal_en_create")
    return ctx


def ssnal_en_destroy(ctx):
    load_library().ssnal_en_destroy(ctx)


def ssnal_en_set_options(ctx, options: Options | None):
    _check(load_library().ssnal_en_set_options(ctx, ctypes.byref(options) if options is not None else None),
           "ssnal_en_set_options")


def ssnal_en_solve(ctx, b, lambda1, lambda2, x, y=None):
    """b, x (in/out), y (optional in/out): FP64 device tensors.  Returns (status, Result)."""
    res = Result()
    st = load_library().ssnal_en_solve(ctx, _ptr(b), float(lambda1), float(lambda2), _ptr(x), _ptr(y),
                                       ctypes.byref(res))
    _check(st, "ssnal_en_solve", allow=(OK, ENOCONV))
    return st, res


def ssnal_en_solve_batch(instances, workers: int = 0):
    """instances: sequence of (ctx, b, lambda1, lambda2, x, y-or-None) with FP64 device tensors.
    Returns (status, [Result], workers_used)."""
    arr = (Instance * len(instances))()
    for k, (ctx, b, l1, l2, x, y) in enumerate(instances):
        arr[k] = Instance(ctx, _ptr(b), float(l1), float(l2), _ptr(x), _ptr(y))
    res = (Result * len(instances))()
    used = ctypes.c_int32(0)
    st = load_library().ssnal_en_solve_batch(arr, len(instances), int(workers), res, ctypes.byref(used))
    _check(st, "ssnal_en_solve_batch", allow=(OK, ENOCONV))
    return st, list(res), used.value


def ssnal_en_solve_shared(instances):
    """Fits whose contexts share one matrix, advanced together with merged passes over A.
    instances: sequence of (ctx, b, lambda1, lambda2, x, y-or-None) with FP64 device tensors.
    Returns (status, [Result], passes over A of the Newton steps)."""
    arr = (Instance * len(instances))()
    for k, (ctx, b, l1, l2, x, y) in enumerate(instances):
        arr[k] = Instance(ctx, _ptr(b), float(l1), float(l2), _ptr(x), _ptr(y))
    res = (Result * len(instances))()
    passes = ctypes.c_int32(0)
    st = load_library().ssnal_en_solve_shared(arr, len(instances), res, ctypes.byref(passes))
    _check(st, "ssnal_en_solve_shared", allow=(OK, ENOCONV))
    return st, list(res), passes.value


def ssnal_en_solve_batch_resident(fits, options: Options | None = None, stream=None):
    """fits: sequence of (A (device tensor (n, lda) float32, column-major A), m, b, lambda1, lambda2, x)
    with b, x FP64 device tensors.  Returns (status, [Result], (loads in flight chosen, fits solved
    again on the regular path))."""
    arr = (BatchFit * len(fits))()
    for k, (A, m, b, l1, l2, x) in enumerate(fits):
        arr[k] = BatchFit(A.data_ptr(), int(m), A.shape[0], A.shape[1], _ptr(b), float(l1), float(l2), _ptr(x))
    res = (Result * len(fits))()
    info = (ctypes.c_int32 * 2)()
    st = load_library().ssnal_en_solve_batch_resident(arr, len(fits), ctypes.byref(options) if options else None,
                                                      res, info, _stream_handle(stream))
    _check(st, "ssnal_en_solve_batch_resident", allow=(OK, ENOCONV))
    return st, list(res), (info[0], info[1])


def ssnal_en_server_set_group(srv, max_group: int):
    _check(load_library().ssnal_en_server_set_group(srv, int(max_group)), "ssnal_en_server_set_group")


def ssnal_en_server_create(mats, workers=8, options: Options | None = None, max_bytes=0):
    """mats: list of (device tensor (n, lda), m, dtype, col_mean, col_scale).  Returns a handle."""
    arr = (Matrix * len(mats))()
    for k, (A, m, dtype, cm, cs) in enumerate(mats):
        lda = A.shape[1] * 4 if dtype == I2_GENO else A.shape[1]
        arr[k] = Matrix(m=m, n=A.shape[0], lda=lda, dtype=dtype, reserved=0, data=A.data_ptr(),
                        col_mean=cm.data_ptr() if cm is not None else None,
                        col_scale=cs.data_ptr() if cs is not None else None)
    h = ctypes.c_void_p()
    _check(load_library().ssnal_en_server_create(ctypes.byref(h), arr, len(mats),
                                                  ctypes.byref(options) if options else None, int(workers),
                                                  int(max_bytes)), "ssnal_en_server_create")
    return h


def ssnal_en_server_submit(srv, mat, b_host, lambda1, lambda2) -> int:
    b = np.ascontiguousarray(b_host, dtype=np.float64)
    t = ctypes.c_int64(0)
    _check(load_library().ssnal_en_server_submit(srv, int(mat), b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                  float(lambda1), float(lambda2), ctypes.byref(t)),
           "ssnal_en_server_submit")
    return t.value


def ssnal_en_server_submit_scaled(srv, mat, b_host, alpha, c) -> int:
    b = np.ascontiguousarray(b_host, dtype=np.float64)
    t = ctypes.c_int64(0)
    _check(load_library().ssnal_en_server_submit_scaled(srv, int(mat),
                                                         b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                         float(alpha), float(c), ctypes.byref(t)),
           "ssnal_en_server_submit_scaled")
    return t.value


def ssnal_en_server_poll(srv, ticket, n, wait=True):
    """Returns None if not done, else (x (n,), Result, (t_submit, t_start, t_done))."""
    x = np.empty(n, dtype=np.float64)
    res = Result()
    times = (ctypes.c_double * 3)()
    done = ctypes.c_int32(0)
    _check(load_library().ssnal_en_server_poll(srv, int(ticket), int(bool(wait)),
                                                x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                ctypes.byref(res), times, ctypes.byref(done)),
           "ssnal_en_server_poll")
    if not done.value:
        return None
    return x, res, tuple(times)


def ssnal_en_server_destroy(srv):
    load_library().ssnal_en_server_destroy(srv)


class Server:
    """Serving loop over resident matrices.  ``mats`` as for ssnal_en_server_create; the
    device tensors must stay alive for the server's lifetime."""

    def __init__(self, mats, workers=8, options: Options | None = None, max_bytes=0, group: int | None = None):
        self._keep = mats
        self.n = [A.shape[0] for A, _, _, _, _ in mats]
        self.h = ssnal_en_server_create(mats, workers, options, max_bytes)
        if group is not None:
            ssnal_en_server_set_group(self.h, group)

    def submit(self, mat, b_host, lambda1, lambda2) -> int:
        return ssnal_en_server_submit(self.h, mat, b_host, lambda1, lambda2)

    def submit_scaled(self, mat, b_host, alpha, c) -> int:
        return ssnal_en_server_submit_scaled(self.h, mat, b_host, alpha, c)

    def poll(self, ticket, mat, wait=True):
        return ssnal_en_server_poll(self.h, ticket, self.n[mat], wait)

    def close(self):
        if getattr(self, "h", None):
            ssnal_en_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ssnal_en_tune(ctx, b, alpha, c_grid, X):
    """Path plus gcv / e-bic at each point (Sec. 3.3).  X: FP64 device tensor (K, n).
    Returns (status, [Result], [TunePoint], best_gcv, best_ebic, n_done)."""
    grid = np.ascontiguousarray(c_grid, dtype=np.float64)
    K = len(grid)
    res = (Result * max(K, 1))()
    crit = (TunePoint * max(K, 1))()
    bg, be, done = ctypes.c_int32(-1), ctypes.c_int32(-1), ctypes.c_int32(0)
    st = load_library().ssnal_en_tune(ctx, _ptr(b), float(alpha), grid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      K, _ptr(X), res, crit, ctypes.byref(bg), ctypes.byref(be), ctypes.byref(done))
    _check(st, "ssnal_en_tune", allow=(OK, ENOCONV))
    return st, list(res)[:done.value], list(crit)[:done.value], bg.value, be.value, done.value


def ssnal_en_path(ctx, b, alpha, c_grid, X=None):
    """b: device FP64 (m); c_grid: host sequence; X: device FP64 (K, n) or None.
    Returns (status, [Result], n_done)."""
    K = len(c_grid)
    cg = (ctypes.c_double * K)(*[float(c) for c in c_grid])
    out = (Result * K)()
    done = ctypes.c_int32(0)
    st = load_library().ssnal_en_path(ctx, _ptr(b), float(alpha), cg, K, _ptr(X), out, ctypes.byref(done))
    _check(st, "ssnal_en_path", allow=(OK, ENOCONV))
    return st, list(out), done.value


def ssnal_en_path_host(ctx, b_host: np.ndarray, alpha, c_grid, X_host: np.ndarray | None = None):
    """b_host: host float64 (m); X_host: host float64 (K, n) or None (written in place)."""
    K = len(c_grid)
    cg = (ctypes.c_double * K)(*[float(c) for c in c_grid])
    out = (Result * K)()
    done = ctypes.c_int32(0)
    b_host = np.ascontiguousarray(b_host, dtype=np.float64)
    bp = b_host.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    xp = None
    if X_host is not None:
        assert X_host.dtype == np.float64 and X_host.flags.c_contiguous
        xp = ctypes.c_void_p(X_host.ctypes.data)
    st = load_library().ssnal_en_path_host(ctx, bp, float(alpha), cg, K, xp, out, ctypes.byref(done))
    _check(st, "ssnal_en_path_host", allow=(OK, ENOCONV))
    return st, list(out), done.value


def ssnal_en_op_at_y(ctx, y, u):
    _check(load_library().ssnal_en_op_at_y(ctx, _ptr(y), _ptr(u)), "ssnal_en_op_at_y")


def ssnal_en_op_at_d(ctx, d, t):
    _check(load_library().ssnal_en_op_at_d(ctx, _ptr(d), _ptr(t)), "ssnal_en_op_at_d")


def ssnal_en_op_prox_active(ctx, x, u, sigma, lambda1, lambda2, J, wJ) -> int:
    r = ctypes.c_int64(0)
    _check(load_library().ssnal_en_op_prox_active(ctx, _ptr(x), _ptr(u), float(sigma), float(lambda1),
                                                  float(lambda2), _ptr(J), _ptr(wJ), ctypes.byref(r)),
           "ssnal_en_op_prox_active")
    return r.value


def ssnal_en_op_grad(ctx, J, wJ, r, y, b, g):
    _check(load_library().ssnal_en_op_grad(ctx, _ptr(J), _ptr(wJ), int(r), _ptr(y), _ptr(b), _ptr(g)),
           "ssnal_en_op_grad")


def ssnal_en_op_newton(ctx, r, kappa, g, d):
    return _check(load_library().ssnal_en_op_newton(ctx, int(r), float(kappa), _ptr(g), _ptr(d)),
                  "ssnal_en_op_newton", allow=(OK, ENOCONV))


PHASES = ("prox_gather_grad", "newton_direction", "stream_line_search", "al_update", "u_refresh")
PROFILE_PHASES = 5  # SSNAL_EN_PROFILE_PHASES


def ssnal_en_profile_phases(ctx):
    """Device ms and counts per phase (see PHASES) since the last profile reset."""
    ms = (ctypes.c_double * PROFILE_PHASES)()
    n = (ctypes.c_int64 * PROFILE_PHASES)()
    _check(load_library().ssnal_en_profile_phases(ctx, ms, n), "ssnal_en_profile_phases")
    return {PHASES[k]: (ms[k], n[k]) for k in range(PROFILE_PHASES)}


def ssnal_en_profile(ctx, enable, reset: bool = False, phases: bool = False):
    """Returns dict(stream_ms, stream_launches, stream_bytes, kernel_launches) of the
    A^T d stream launches that carried events: one in eight at level 1; every
    launch, and the phases of ssnal_en_profile_phases, with ``phases`` (level 2)."""
    ms, nl, by, kl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
    level = (2 if phases else 1) if enable else 0
    _check(load_library().ssnal_en_profile(ctx, level, int(bool(reset)), ctypes.byref(ms),
                                           ctypes.byref(nl), ctypes.byref(by), ctypes.byref(kl)),
           "ssnal_en_profile")
    return {"stream_ms": ms.value, "stream_launches": nl.value, "stream_bytes": by.value,
            "kernel_launches": kl.value}


def ssnal_en_prox_active_static(x, u, sigma, lambda1, lambda2, J, wJ, stream=None) -> int:
    """Allocation-free prox / active-set step (no context; see the header for the
    limits and the shared-scratch rules).  x, u: FP64 device tensors of length n on the
    current device; J (int32), wJ (FP64): device outputs of capacity n.  Synchronous:
    do not call it while the stream is being captured.  Returns |J|."""
    import torch
    n = int(x.numel())
    for name, t, dt in (("x", x, torch.float64), ("u", u, torch.float64), ("J", J, torch.int32),
                        ("wJ", wJ, torch.float64)):
        if t.dtype != dt or not t.is_contiguous() or t.device.type != "cuda":
            raise ValueError(f"ssnal_en_prox_active_static: {name} must be a contiguous CUDA {dt} tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"ssnal_en_prox_active_static: {name} is on {t.device}, the current device is "
                             f"cuda:{torch.cuda.current_device()} (the scratch address is per device)")
    if u.numel() != n or J.numel() < n or wJ.numel() < n:
        raise ValueError("ssnal_en_prox_active_static: u needs n entries, J and wJ at least n")
    r = ctypes.c_int64(0)
    _check(load_library().ssnal_en_prox_active_static(_ptr(x), _ptr(u), n, float(sigma),
                                                      float(lambda1), float(lambda2), _ptr(J), _ptr(wJ),
                                                      ctypes.byref(r), _stream_handle(stream)),
           "ssnal_en_prox_active_static")
    return r.value


class Context:
    """Owns one library context for a resident design matrix.

    ``At`` is the feature-major (n, m) host array (== column-major A), or an
    already padded device tensor together with ``m``.
    """

    def __init__(self, At, m: int | None = None, dtype: int = F64, options: Options | None = None, stream=None,
                 col_mean=None, col_scale=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("SsNAL-EN needs a CUDA device; there is no CPU fallback")
        if isinstance(At, np.ndarray):
            self.A, self.m = device_matrix(At, dtype)
        else:
            self.A, self.m = At, int(m)
        self.n = self.A.shape[0]
        self.dtype = dtype
        self._keep = (col_mean, col_scale)
        self.ctx = ssnal_en_create(self.A, self.m, dtype, options, stream, col_mean, col_scale)

    def close(self):
        if getattr(self, "ctx", None):
            ssnal_en_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, options):
        ssnal_en_set_options(self.ctx, options)

    def solve(self, b, lambda1, lambda2, x0=None, y=None):
        import torch
        b = torch.as_tensor(b, dtype=torch.float64, device="cuda")
        x = torch.zeros(self.n, dtype=torch.float64, device="cuda") if x0 is None else \
            torch.as_tensor(x0, dtype=torch.float64, device="cuda").clone()
        y = torch.zeros(self.m, dtype=torch.float64, device="cuda") if y is None else y
        st, res = ssnal_en_solve(self.ctx, b, lambda1, lambda2, x, y)
        return x, y, res

    def path(self, b, alpha, c_grid, keep_X=True):
        import torch
        b = torch.as_tensor(b, dtype=torch.float64, device="cuda")
        X = torch.zeros((len(c_grid), self.n), dtype=torch.float64, device="cuda") if keep_X else None
        st, res, done = ssnal_en_path(self.ctx, b, alpha, c_grid, X)
        return X, res, done
