"""Pins for Prop. 2, eq. grad_phy and the Newton system (Sec. 3.1-3.2)."""
import numpy as np
import pytest

from oracle import ssnal_en_ref as R
from paper_2006_03970_gb300 import synth


def _case(m=30, n=80, seed=3, sigma=0.7):
    p = synth.make_problem(m, n, k=6, seed=seed, alpha=0.7)
    l1, l2 = R.lambdas(p.At, p.b, 0.7, 0.4)
    rng = np.random.default_rng(seed)
    x = rng.normal(size=n) * (rng.random(n) < 0.2)
    y = rng.normal(size=m) * 2
    return p.At, p.b, x, y, sigma, l1, l2


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_psi_equals_lagrangian_at_z_bar(seed):
    At, b, x, y, s, l1, l2 = _case(seed=seed)
    z = R.z_bar(y, x, At, s, l1, l2)
    assert R.psi(y, x, At, b, s, l1, l2) == pytest.approx(R.aug_lagrangian(y, z, x, At, b, s, l1, l2), rel=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_z_bar_minimises_lagrangian(seed):
    At, b, x, y, s, l1, l2 = _case(seed=seed)
    z = R.z_bar(y, x, At, s, l1, l2)
    L0 = R.aug_lagrangian(y, z, x, At, b, s, l1, l2)
    rng = np.random.default_rng(seed + 10)
    for scale in [1e-1, 1e-3, 1e-5]:
        for _ in range(5):
            dz = rng.normal(size=z.size) * scale
            assert R.aug_lagrangian(y, z + dz, x, At, b, s, l1, l2) >= L0 - 1e-12 * abs(L0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grad_psi_central_differences(seed):
    At, b, x, y, s, l1, l2 = _case(seed=seed)
    g = R.grad_psi(y, x, At, b, s, l1, l2)
    h = 1e-6
    fd = np.array([(R.psi(y + h * e, x, At, b, s, l1, l2) - R.psi(y - h * e, x, At, b, s, l1, l2)) / (2 * h)
                   for e in np.eye(y.size)])
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())


@pytest.mark.parametrize("seed", [0, 1])
def test_generalized_hessian_directional_derivative(seed):
    # Away from kinks, grad psi is piecewise affine and its derivative along d is V d,
    # V = I + sigma A Q A^T with Q from eq. Q_def.
    At, b, x, y, s, l1, l2 = _case(seed=seed)
    v = x - s * (At @ y)
    J = R.active_set(v, s, l1)
    kappa = s / (1 + s * l2)
    d = np.random.default_rng(seed).normal(size=y.size)
    h = 1e-7
    assert np.all(np.abs(np.abs(v) - s * l1) > 1e-4)
    Vd = d + kappa * At[J].T @ (At[J] @ d)
    fd = (R.grad_psi(y + h * d, x, At, b, s, l1, l2) - R.grad_psi(y - h * d, x, At, b, s, l1, l2)) / (2 * h)
    np.testing.assert_allclose(fd, Vd, rtol=1e-6, atol=1e-6 * np.abs(Vd).max())


@pytest.mark.parametrize("r", [0, 1, 7, 29, 30, 31, 55])
def test_smw_matches_direct_solve(r):
    m = 30
    rng = np.random.default_rng(r)
    AJt = rng.normal(size=(r, m))
    g = rng.normal(size=m)
    kappa = 0.37
    d = R.newton_direction(AJt, g, kappa)
    V = np.eye(m) + kappa * AJt.T @ AJt
    np.testing.assert_allclose(V @ d, -g, rtol=1e-11, atol=1e-11)


def test_newton_direction_is_descent():
    At, b, x, y, s, l1, l2 = _case(seed=5)
    g = R.grad_psi(y, x, At, b, s, l1, l2)
    v = x - s * (At @ y)
    J = R.active_set(v, s, l1)
    d = R.newton_direction(At[J], g, s / (1 + s * l2))
    assert g @ d < 0
