"""The checkers that pin the oracle are themselves checked against each other and against a
library optimiser (L-BFGS-B on the split form x = x+ - x-), so that none of them can carry a
mistake of its own into the pins."""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import checkers as C
from paper_2006_03970_gb300 import synth


def _lbfgsb(At, b, lam1, lam2):
    # min 1/2 ||A (p - q) - b||^2 + lam1 sum(p + q) + lam2/2 ||p - q||^2 over p, q >= 0: the
    # Elastic Net objective with its minimiser at p - q (smooth, bound constrained)
    n = At.shape[0]

    def f(z):
        p, q = z[:n], z[n:]
        x = p - q
        r = At.T @ x - b
        g = At @ r + lam2 * x
        val = 0.5 * (r @ r) + lam1 * (p.sum() + q.sum()) + 0.5 * lam2 * (x @ x)
        return val, np.concatenate([g + lam1, -g + lam1])

    res = minimize(f, np.zeros(2 * n), jac=True, method="L-BFGS-B", bounds=[(0, None)] * (2 * n),
                   options={"maxiter": 20000, "ftol": 1e-15, "gtol": 1e-12, "maxcor": 30})
    return res.x[:n] - res.x[n:]


def _problem(m, n, seed, alpha, c):
    p = synth.make_problem(m, n, k=min(4, n), seed=seed, snr=3.0, block=4, rho=0.4)
    g = np.abs(p.At @ p.b).max()
    return p, c * g, (1 - alpha) / alpha * c * g


@pytest.mark.parametrize("seed", range(4))
def test_brute_force_and_coordinate_descent_agree(seed):
    p, l1, l2 = _problem(8 + seed, 7, 200 + seed, 0.7, [0.1, 0.3, 0.6, 0.05][seed])
    xb = C.brute_force(p.At, p.b, l1, l2)
    xc = C.coordinate_descent(p.At, p.b, l1, l2)
    np.testing.assert_allclose(xc, xb, atol=1e-10 * max(1.0, np.abs(xb).max()))


@pytest.mark.parametrize("seed", range(3))
def test_coordinate_descent_and_lbfgsb_agree(seed):
    p, l1, l2 = _problem(40, 120, 300 + seed, 0.6, 0.2)
    xc = C.coordinate_descent(p.At, p.b, l1, l2)
    xl = _lbfgsb(p.At, p.b, l1, l2)
    Pc, Pl = C.primal_objective(p.At, p.b, xc, l1, l2), C.primal_objective(p.At, p.b, xl, l1, l2)
    assert Pc <= Pl + 1e-10 * Pl  # coordinate descent is at least as good as the library optimiser
    assert np.abs(xc - xl).max() <= 1e-5 * np.abs(xc).max()


def test_kkt_violation_and_duality_gap_vanish_only_at_the_minimiser():
    p, l1, l2 = _problem(50, 200, 7, 0.8, 0.3)
    x = C.coordinate_descent(p.At, p.b, l1, l2)
    y = p.At.T @ x - p.b
    assert C.kkt_violation(p.At, p.b, x, l1, l2) <= 1e-10
    P, D = C.primal_objective(p.At, p.b, x, l1, l2), C.dual_objective(p.At, p.b, y, l1, l2)
    assert abs(P - D) <= 1e-10 * abs(P)
    x2 = x.copy()
    x2[np.flatnonzero(x)[0]] *= 1.01
    y2 = p.At.T @ x2 - p.b
    assert C.kkt_violation(p.At, p.b, x2, l1, l2) > 1e-6
    assert C.primal_objective(p.At, p.b, x2, l1, l2) - C.dual_objective(p.At, p.b, y2, l1, l2) > 1e-9 * abs(P)


def test_weak_duality_everywhere():
    p, l1, l2 = _problem(30, 60, 8, 0.5, 0.4)
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = rng.normal(size=60) * (rng.random(60) < 0.3)
        y = rng.normal(size=30) * 3
        assert C.primal_objective(p.At, p.b, x, l1, l2) >= C.dual_objective(p.At, p.b, y, l1, l2)


def test_closed_forms_match_coordinate_descent():
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.normal(size=(40, 12)))
    At = (Q * rng.uniform(0.5, 2.0, 12)).T.copy()  # 12 orthogonal columns of different norms
    b = rng.normal(size=40)
    for l1, l2 in [(0.3, 0.2), (1.0, 0.0), (0.05, 3.0)]:
        np.testing.assert_allclose(C.orthogonal_closed_form(At, b, l1, l2),
                                   C.coordinate_descent(At, b, l1, l2), atol=1e-12)
    p = synth.make_problem(30, 20, k=4, seed=10)
    np.testing.assert_allclose(C.ridge_closed_form(p.At, p.b, 0.7), C.coordinate_descent(p.At, p.b, 0.0, 0.7),
                               rtol=1e-9, atol=1e-11)
