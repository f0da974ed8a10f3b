"""Pins for the convex-analysis primitives of the oracle (Sec. 2): Prop. 1 and eq. prox_elastic
checked against their definitions (numerical sup / argmin), and the Moreau decomposition."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import ssnal_en_ref as R

PARAMS = [(1.0, 1.0, 1.0), (0.3, 2.5, 0.7), (2.0, 0.1, 5e-3), (0.05, 4.0, 40.0)]


def _pen1(x, l1, l2):
    return l1 * abs(x) + 0.5 * l2 * x * x


@pytest.mark.parametrize("l1,l2,_s", PARAMS)
def test_p_star_is_the_conjugate(l1, l2, _s):
    # p*(z) = sup_x (z x - p(x)) in 1-D (Prop. 1); the sup is attained in [-B, B].
    for z in [-3.7 * l1, -l1 - 0.2, -l1, -0.5 * l1, 0.0, 0.9 * l1, l1, l1 + 1e-3, 2.2 * l1 + 1.0]:
        res = minimize_scalar(lambda x: -(z * x - _pen1(x, l1, l2)), bounds=(-1e3, 1e3), method="bounded",
                              options={"xatol": 1e-12})
        sup = -res.fun
        assert R.p_star(np.array([z]), l1, l2) == pytest.approx(sup, abs=1e-9, rel=1e-9)


def test_p_star_separable_sum():
    rng = np.random.default_rng(1)
    z = rng.normal(size=17) * 3
    l1, l2 = 0.7, 1.9
    tot = sum(R.p_star(np.array([zi]), l1, l2) for zi in z)
    assert R.p_star(z, l1, l2) == pytest.approx(tot, rel=1e-14)


@pytest.mark.parametrize("l1,l2,s", PARAMS)
def test_prox_sigma_p_is_argmin(l1, l2, s):
    # prox_{s p}(x) = argmin_t p(t) + (2s)^{-1} (t - x)^2 (eq. prox_op, eq. prox_elastic).
    for x in np.linspace(-4 * s * l1 - 1, 4 * s * l1 + 1, 23):
        res = minimize_scalar(lambda t: _pen1(t, l1, l2) + (t - x) ** 2 / (2 * s), bracket=(-50, 50),
                              method="brent", tol=1e-14)
        assert R.prox_sigma_p(np.array([x]), s, l1, l2)[0] == pytest.approx(res.x, abs=1e-7)


@pytest.mark.parametrize("l1,l2,s", PARAMS)
def test_prox_p_star_is_argmin(l1, l2, s):
    # prox_{p*/s}(t/s) = argmin_z p*(z)/s + 1/2 (z - t/s)^2, i.e. the prox of (1/s) p*.
    for t in np.linspace(-3 * s * l1 - 2, 3 * s * l1 + 2, 19):
        f = lambda z: R.p_star(np.array([z]), l1, l2) / s + 0.5 * (z - t / s) ** 2
        res = minimize_scalar(f, bracket=(-100, 100), method="brent", tol=1e-14)
        assert R.prox_p_star_over_sigma(np.array([t]), s, l1, l2)[0] == pytest.approx(res.x, abs=1e-6, rel=1e-7)


@pytest.mark.parametrize("l1,l2,s", PARAMS)
def test_moreau_decomposition(l1, l2, s):
    # t = prox_{s p}(t) + s prox_{p*/s}(t/s) (Sec. 2.2).
    t = np.linspace(-10, 10, 2001) * max(1.0, s * l1)
    lhs = R.prox_sigma_p(t, s, l1, l2) + s * R.prox_p_star_over_sigma(t, s, l1, l2)
    np.testing.assert_allclose(lhs, t, rtol=1e-13, atol=1e-13 * max(1, s * l1))


def test_fig1_setting_values():
    # lam1 = lam2 = sigma = 1 (the setting of Fig. 1): p*(z) = (|z|-1)_+^2 / 2,
    # prox_{p}(x) = soft(x, 1) / 2, prox_{p*}(x) = x for |x| < 1 and (x +- 1)/2 outside.
    z = np.array([-3.0, -1.0, -0.4, 0.0, 0.6, 1.0, 2.5])
    for zi in z:
        assert R.p_star(np.array([zi]), 1, 1) == pytest.approx(0.5 * max(abs(zi) - 1, 0) ** 2)
    np.testing.assert_allclose(R.prox_sigma_p(z, 1, 1, 1), [-1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.75])
    np.testing.assert_allclose(R.prox_p_star_over_sigma(z, 1, 1, 1), [-2.0, -1.0, -0.4, 0.0, 0.6, 1.0, 1.75])
