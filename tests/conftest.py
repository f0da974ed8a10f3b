import os
import sys

# The oracle's dense solves run on one BLAS thread in the test-suite, so that a
# result cannot depend on how a threaded BLAS splits the work or on the machine's
# load.  Set before NumPy / SciPy load their OpenBLAS, and again on the loaded
# libraries below (in case a plugin imported NumPy first).
for _k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
    os.environ[_k] = "1"

import pytest  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import blas as _blas  # noqa: E402

_blas.set_blas_threads(1)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running oracle case")


def pytest_report_header(config):
    return "oracle BLAS threads: " + ", ".join(f"{k}={v}" for k, v in sorted(_blas.blas_threads().items()))
