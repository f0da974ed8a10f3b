"""Pins of the tuning criteria of the oracle (Sec. 3.3, eq. gcv_bic) against closed forms."""
import numpy as np
import pytest

from oracle import ssnal_en_ref as R


def orthonormal_columns(m, n, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(m, n)))
    return q.T.copy()  # At (n, m) with orthonormal rows = orthonormal columns of A


@pytest.mark.parametrize("lam2", [0.0, 0.3, 2.0])
def test_degrees_of_freedom_orthonormal(lam2):
    # A_J^T A_J = I: nu = r / (1 + lam2)
    At = orthonormal_columns(30, 12, 1)
    x = np.zeros(12)
    x[[0, 3, 4, 9]] = [1.0, -2.0, 0.5, 3.0]
    assert R.en_degrees_of_freedom(At, x, lam2) == pytest.approx(4 / (1 + lam2), rel=1e-12)


def test_degrees_of_freedom_spectrum():
    # nu = sum_i s_i^2 / (s_i^2 + lam2) over the singular values of A_J, also when r > m
    rng = np.random.default_rng(2)
    At = rng.normal(size=(40, 15))
    x = np.zeros(40)
    x[rng.choice(40, size=22, replace=False)] = 1.0
    s = np.linalg.svd(At[np.flatnonzero(x)].T, compute_uv=False)
    lam2 = 0.7
    assert R.en_degrees_of_freedom(At, x, lam2) == pytest.approx(np.sum(s**2 / (s**2 + lam2)), rel=1e-10)
    assert R.en_degrees_of_freedom(At, np.zeros(40), lam2) == 0.0


def test_debiased_rss_orthonormal_and_interpolation():
    At = orthonormal_columns(25, 10, 3)
    b = np.random.default_rng(4).normal(size=25)
    x = np.zeros(10)
    x[[1, 2, 7]] = 1.0
    proj = At[[1, 2, 7]] @ b
    assert R.debiased_rss(At, b, x) == pytest.approx(b @ b - proj @ proj, rel=1e-12)
    # r >= m generic: least squares interpolates
    rng = np.random.default_rng(5)
    At2 = rng.normal(size=(30, 8))
    x2 = np.ones(30)
    assert R.debiased_rss(At2, rng.normal(size=8), x2) == pytest.approx(0.0, abs=1e-18)


def test_criteria_formulas():
    rng = np.random.default_rng(6)
    At = rng.normal(size=(50, 20))
    b = rng.normal(size=20)
    x = np.zeros(50)
    x[[3, 8, 11]] = 1.0
    nu, rss, gcv, ebic = R.tuning_criteria(At, b, x, 0.5)
    m, n = 20, 50
    assert gcv == pytest.approx(rss / m / (1 - nu / m) ** 2, rel=1e-14)
    assert ebic == pytest.approx(np.log(rss / m) + nu / m * (np.log(m) + np.log(n)), rel=1e-14)
    assert 0 < nu < 3
