"""Thread count of the BLAS / LAPACK libraries the oracle runs on (test infrastructure only).

NumPy and SciPy each load their own OpenBLAS.  The oracle's small dense solves are
written to be exact to FP64 rounding, so the test-suite runs them on one BLAS thread:
the result of a solve then cannot depend on how a threaded BLAS splits its work or
on the load of the machine.  The CPU-baseline leg of the benchmark may raise the
count to the host's cores (and reports the count it used).

``set_blas_threads(n)`` sets the count of every OpenBLAS loaded in this process,
through threadpoolctl where it is installed, else through each library's own
``*_set_num_threads`` entry point found by scanning the process's mapped libraries.
``blas_threads()`` reports the counts.  Importing NumPy / SciPy first is the caller's
business; the environment variables set by ``pin_env`` only affect libraries that
are loaded after the call.
"""
from __future__ import annotations

import ctypes
import os

_ENV_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")
_SETTERS = ("scipy_openblas_set_num_threads64_", "scipy_openblas_set_num_threads", "openblas_set_num_threads64_",
            "openblas_set_num_threads")
_GETTERS = ("scipy_openblas_get_num_threads64_", "scipy_openblas_get_num_threads", "openblas_get_num_threads64_",
            "openblas_get_num_threads")


def pin_env(n: int = 1) -> None:
    """Thread-count variables for BLAS libraries that are not loaded yet."""
    for k in _ENV_VARS:
        os.environ[k] = str(int(n))


def _loaded_openblas():
    paths = []
    try:
        with open("/proc/self/maps") as f:
            for line in f:
                p = line.split()[-1]
                if "openblas" in os.path.basename(p) and ".so" in p and p not in paths:
                    paths.append(p)
    except OSError:
        pass
    return paths


def _ctypes_libs():
    out = []
    for p in _loaded_openblas():
        try:
            lib = ctypes.CDLL(p)
        except OSError:
            continue
        setter = next((getattr(lib, s) for s in _SETTERS if hasattr(lib, s)), None)
        getter = next((getattr(lib, g) for g in _GETTERS if hasattr(lib, g)), None)
        if setter is not None:
            out.append((p, setter, getter))
    return out


def set_blas_threads(n: int) -> int:
    """Sets the thread count of every loaded OpenBLAS to n; returns how many libraries
    were set."""
    import numpy  # noqa: F401  (load both BLAS libraries before setting them)
    import scipy.linalg  # noqa: F401
    try:
        import threadpoolctl
        threadpoolctl.threadpool_limits(limits=int(n), user_api="blas")
        return len([i for i in threadpoolctl.threadpool_info() if i.get("user_api") == "blas"])
    except ImportError:
        pass
    libs = _ctypes_libs()
    for _, setter, _ in libs:
        setter.argtypes = [ctypes.c_int]
        setter.restype = None
        setter(int(n))
    return len(libs)


def blas_threads() -> dict:
    """{library file: thread count} of the loaded OpenBLAS libraries (-1 if unknown)."""
    out = {}
    try:
        import threadpoolctl
        for i in threadpoolctl.threadpool_info():
            if i.get("user_api") == "blas":
                out[os.path.basename(i["filepath"])] = int(i["num_threads"])
        return out
    except ImportError:
        pass
    for p, _, getter in _ctypes_libs():
        if getter is None:
            out[os.path.basename(p)] = -1
            continue
        getter.argtypes = []
        getter.restype = ctypes.c_int
        out[os.path.basename(p)] = int(getter())
    return out
