"""Pins for the whole SsNAL-EN oracle solution against checkers that do not use the method:
brute force, coordinate descent, closed forms, KKT conditions and the duality gap."""
import numpy as np
import pytest

from oracle import checkers as C
from oracle import ssnal_en_ref as R
from paper_2006_03970_gb300 import synth

TIGHT = R.Options(tol=1e-9, max_al=200)  # below ~1e-10 the Armijo test of eq. line_search drowns in FP64 rounding of psi


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_tiny(seed):
    m, n = 6 + seed, 6 + (seed % 3)
    p = synth.make_problem(m, n, k=3, seed=100 + seed, snr=3.0)
    c = [0.15, 0.3, 0.5, 0.7, 0.05, 0.9][seed]
    l1, l2 = R.lambdas(p.At, p.b, 0.7, c)
    xb = C.brute_force(p.At, p.b, l1, l2)
    r = R.solve(p.At, p.b, l1, l2, opts=TIGHT)
    assert r.converged
    np.testing.assert_allclose(r.x, xb, atol=1e-7 * max(1, np.abs(xb).max()))
    assert np.array_equal(np.flatnonzero(r.x), np.flatnonzero(xb))


@pytest.mark.parametrize("m,n,alpha,c,seed", [(50, 200, 0.8, 0.3, 0), (100, 2000, 0.8, 0.5, 0),
                                              (40, 300, 0.5, 0.1, 7), (120, 600, 0.95, 0.2, 8)])
def test_coordinate_descent(m, n, alpha, c, seed):
    p = synth.make_problem(m, n, k=10, seed=seed, block=10, rho=0.5)
    l1, l2 = R.lambdas(p.At, p.b, alpha, c)
    xc = C.coordinate_descent(p.At, p.b, l1, l2)
    r = R.solve(p.At, p.b, l1, l2, opts=TIGHT)
    assert r.converged
    assert np.abs(r.x - xc).max() <= 1e-7 * np.abs(xc).max()
    assert np.array_equal(np.flatnonzero(r.x), np.flatnonzero(xc))


def test_config1_default_tolerance_is_within_tolerance_of_cd():
    p = synth.config1()
    l1, l2 = R.lambdas(p.At, p.b, p.alpha, p.c)
    r = R.solve(p.At, p.b, l1, l2)
    xc = C.coordinate_descent(p.At, p.b, l1, l2)
    assert r.converged and 2 <= r.al_iters <= 6
    assert np.abs(r.x - xc).max() <= 1e-5 * np.abs(xc).max()
    P = C.primal_objective(p.At, p.b, r.x, l1, l2)
    assert abs(P - C.primal_objective(p.At, p.b, xc, l1, l2)) <= 1e-10 * P


@pytest.mark.parametrize("c", [1.0, 1.3])
def test_zero_solution_above_threshold(c):
    # lam1 >= ||A^T b||_inf gives x = 0 (Sec. 3.3); then y = A x - b = -b.
    p = synth.make_problem(60, 500, k=5, seed=4)
    l1, l2 = R.lambdas(p.At, p.b, 0.6, c)
    r = R.solve(p.At, p.b, l1, l2)
    assert r.converged and np.all(r.x == 0.0)
    np.testing.assert_array_equal(r.y, -p.b)


def test_just_below_threshold_is_nonzero():
    p = synth.make_problem(60, 500, k=5, seed=4)
    l1, l2 = R.lambdas(p.At, p.b, 0.6, 0.999)
    r = R.solve(p.At, p.b, l1, l2)
    assert np.count_nonzero(r.x) >= 1


@pytest.mark.parametrize("lam2", [1.0, 0.25])
def test_orthonormal_closed_form(lam2):
    rng = np.random.default_rng(9)
    m, n = 40, 25
    Q, _ = np.linalg.qr(rng.normal(size=(m, n)))
    At = np.ascontiguousarray(Q.T)
    b = rng.normal(size=m) * 3
    l1 = 0.8
    expect = C.soft(At @ b, l1) / (1 + lam2)
    r = R.solve(At, b, l1, lam2, opts=TIGHT)
    np.testing.assert_allclose(r.x, expect, atol=1e-8)
    np.testing.assert_allclose(C.orthogonal_closed_form(At, b, l1, lam2), expect, atol=1e-14)


def test_orthogonal_columns_with_norms():
    rng = np.random.default_rng(10)
    m, n = 30, 12
    Q, _ = np.linalg.qr(rng.normal(size=(m, n)))
    At = np.ascontiguousarray(Q.T * rng.uniform(0.5, 3.0, size=n)[:, None])
    b = rng.normal(size=m) * 2
    l1, l2 = 0.5, 0.3
    r = R.solve(At, b, l1, l2, opts=TIGHT)
    np.testing.assert_allclose(r.x, C.orthogonal_closed_form(At, b, l1, l2), atol=1e-8)


def test_ridge_when_lam1_zero():
    p = synth.make_problem(30, 90, k=5, seed=11)
    lam2 = 2.0
    r = R.solve(p.At, p.b, 0.0, lam2, opts=TIGHT)
    np.testing.assert_allclose(r.x, C.ridge_closed_form(p.At, p.b, lam2), rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("m,n,alpha,c,seed", [(100, 2000, 0.8, 0.5, 0), (150, 4000, 0.6, 0.2, 1)])
def test_kkt_and_duality_gap(m, n, alpha, c, seed):
    p = synth.make_problem(m, n, k=10, seed=seed, block=20, rho=0.7)
    l1, l2 = R.lambdas(p.At, p.b, alpha, c)
    r = R.solve(p.At, p.b, l1, l2)
    assert r.converged and r.kkt1 <= 1e-6 and r.kkt3 <= 1e-6
    assert C.kkt_violation(p.At, p.b, r.x, l1, l2) <= 1e-5
    P = C.primal_objective(p.At, p.b, r.x, l1, l2)
    D = C.dual_objective(p.At, p.b, r.y, l1, l2)
    assert -1e-9 * abs(P) <= P - D <= 1e-6 * abs(P)


@pytest.mark.parametrize("n0,alpha,seed", [(40, 0.6, 0), (10, 0.75, 1), (5, 0.9, 2)])
def test_al_iterations_band(n0, alpha, seed):
    # Sec. 4.1: convergence in no more than 6 AL iterations on sim-like problems.
    p = synth.make_problem(200, 5000, k=n0, seed=seed, lo=5.0, hi=5.0)
    l1, l2 = R.lambdas(p.At, p.b, alpha, 0.5)
    r = R.solve(p.At, p.b, l1, l2)
    assert r.converged and 1 <= r.al_iters <= 6


def test_path_warm_start_matches_cold_and_truncates():
    p = synth.make_problem(80, 800, k=8, seed=12, block=20, rho=0.7)
    grid = synth.path_grid(8, 0.1)
    res = R.path(p.At, p.b, 0.6, grid)
    assert np.all(res[0].x == 0.0)
    for rr in res[1:]:
        xc = C.coordinate_descent(p.At, p.b, rr.lam1, rr.lam2)
        assert np.abs(rr.x - xc).max() <= 1e-4 * max(1e-12, np.abs(xc).max())
    nnz = [np.count_nonzero(rr.x) for rr in res]
    k = next(i for i, v in enumerate(nnz) if v >= 3)
    trunc = R.path(p.At, p.b, 0.6, grid, max_active=3)
    assert len(trunc) == k + 1


def _golden():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "tiny_en.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_golden_tiny(case):
    At = np.ascontiguousarray(np.array(case["A"]).T)
    b = np.array(case["b"])
    r = R.solve(At, b, case["lam1"], case["lam2"], opts=TIGHT)
    assert r.converged
    np.testing.assert_allclose(r.x, case["x"], atol=1e-7 * max(1.0, np.abs(case["x"]).max()))
    assert np.array_equal(np.flatnonzero(r.x), np.flatnonzero(case["x"]))
