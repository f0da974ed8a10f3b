"""Pins for the conjugate-gradient Newton solve of the oracle (Algorithm 1 step (1), Sec. 3.2):
the direct solve, the Krylov bound on the number of iterations (V = I + kappa A_J A_J^T has at
most rank(A_J) + 1 distinct eigenvalues), the monotone V-norm error of CG, the first step as
the exact line minimiser along -g, and whole fits with CG forced on against coordinate
descent."""
import numpy as np
import pytest

from oracle import checkers as C
from oracle import ssnal_en_ref as R
from paper_2006_03970_gb300 import synth


def _system(r, m, seed, kappa=0.37):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(r, m)), rng.normal(size=m), kappa


@pytest.mark.parametrize("r", [0, 1, 7, 29, 30, 31, 55])
def test_cg_matches_direct_solve(r):
    AJt, g, kappa = _system(r, 30, r)
    d, it = R.newton_direction_cg(AJt, g, kappa, rtol=1e-13)
    np.testing.assert_allclose(d, R.newton_direction(AJt, g, kappa), rtol=1e-10, atol=1e-12)
    assert it <= 3 * 30


@pytest.mark.parametrize("r,m", [(0, 50), (1, 50), (3, 200), (12, 300)])
def test_cg_iterations_within_the_krylov_bound(r, m):
    # V has the eigenvalue 1 on the complement of range(A_J) and rank(A_J) others: CG ends in at
    # most rank + 1 steps in exact arithmetic (one more allowed for rounding)
    AJt, g, kappa = _system(r, m, 100 + r, kappa=0.05)
    d, it = R.newton_direction_cg(AJt, g, kappa, rtol=1e-12)
    assert it <= r + 2
    V = np.eye(m) + kappa * AJt.T @ AJt
    assert np.linalg.norm(V @ d + g) <= 1e-11 * np.linalg.norm(g)
    if r == 0:
        assert it == 1 and np.array_equal(d, -g)


def test_cg_error_decreases_in_the_V_norm():
    # CG minimises the V-norm of the error over nested Krylov spaces
    AJt, g, kappa = _system(40, 60, 7, kappa=2.0)
    V = np.eye(60) + kappa * AJt.T @ AJt
    dstar = np.linalg.solve(V, -g)
    hist = []
    R.newton_direction_cg(AJt, g, kappa, rtol=1e-13, history=hist)
    errs = [np.sqrt((h - dstar) @ V @ (h - dstar)) for h in hist]
    e0 = np.sqrt(dstar @ V @ dstar)
    assert len(errs) >= 5
    assert errs[0] < e0 and all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:]))


def test_cg_first_step_is_the_exact_line_minimiser():
    # the quadratic q(d) = 1/2 d^T V d + g^T d restricted to d = -t g is minimal at
    # t = g^T g / g^T V g
    AJt, g, kappa = _system(9, 40, 3)
    V = np.eye(40) + kappa * AJt.T @ AJt
    hist = []
    R.newton_direction_cg(AJt, g, kappa, maxiter=1, history=hist)
    np.testing.assert_allclose(hist[0], -(g @ g) / (g @ V @ g) * g, rtol=1e-13)


def test_solve_with_cg_forced_on_matches_coordinate_descent():
    p = synth.make_problem(40, 160, k=6, seed=21, block=8, rho=0.5)
    l1, l2 = R.lambdas(p.At, p.b, 0.7, 0.3)
    xc = C.coordinate_descent(p.At, p.b, l1, l2)
    r = R.solve(p.At, p.b, l1, l2, opts=R.Options(tol=1e-8, max_al=60, cg_above=0, cg_rtol=1e-12))
    assert r.converged
    assert np.abs(r.x - xc).max() <= 1e-6 * np.abs(xc).max()
    assert np.array_equal(np.flatnonzero(r.x), np.flatnonzero(xc))


@pytest.mark.parametrize("seed", [0, 1])
def test_fit_with_cg_near_the_switch_matches_the_direct_solve(seed):
    # a lowered threshold sends some Newton steps of one fit to CG and others to the
    # direct solve (r crosses the threshold); both fits meet the KKT tolerance and
    # reach the same objective and support
    p = synth.make_problem(60, 300, k=8, seed=40 + seed, block=10, rho=0.6)
    l1, l2 = R.lambdas(p.At, p.b, 0.6, 0.2)
    direct = R.solve(p.At, p.b, l1, l2, opts=R.Options(tol=1e-8))
    mixed = R.solve(p.At, p.b, l1, l2, opts=R.Options(tol=1e-8, cg_above=50, cg_rtol=1e-12))
    assert max(direct.r_history) > 50 >= min(direct.r_history)  # m = 60: the threshold is crossed
    for res in (direct, mixed):
        assert res.converged and res.kkt1 <= 1e-8 and res.kkt3 <= 1e-8
    Pd = C.primal_objective(p.At, p.b, direct.x, l1, l2)
    Pm = C.primal_objective(p.At, p.b, mixed.x, l1, l2)
    assert abs(Pd - Pm) <= 1e-10 * max(1.0, abs(Pd))
    assert np.abs(direct.x - mixed.x).max() <= 1e-6 * np.abs(direct.x).max()
    assert np.array_equal(np.flatnonzero(direct.x), np.flatnonzero(mixed.x))
