"""The oracle runs on one BLAS thread in the test-suite (oracle.blas), and the
thread-count helper sets and reports every loaded OpenBLAS."""
import numpy as np

from oracle import blas


def test_every_loaded_blas_runs_one_thread():
    counts = blas.blas_threads()
    assert counts, "no OpenBLAS found among the loaded libraries"
    assert all(v == 1 for v in counts.values()), counts


def test_set_blas_threads_round_trip():
    try:
        assert blas.set_blas_threads(2) >= 1
        assert all(v == 2 for v in blas.blas_threads().values())
        a = np.arange(16.0).reshape(4, 4)
        np.testing.assert_array_equal(a @ np.eye(4), a)
    finally:
        blas.set_blas_threads(1)
    assert all(v == 1 for v in blas.blas_threads().values())
