"""The pins must catch plausible mistakes: each case plants one mistake in the oracle
(on the CPU, through monkeypatch) and checks that an independent pin then fails."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import checkers as C
from oracle import ssnal_en_ref as R
from paper_2006_03970_gb300 import synth


def _solution_matches_cd():
    p = synth.make_problem(40, 160, k=6, seed=21, block=8, rho=0.5)
    l1, l2 = R.lambdas(p.At, p.b, 0.7, 0.3)
    xc = C.coordinate_descent(p.At, p.b, l1, l2)
    try:
        r = R.solve(p.At, p.b, l1, l2, opts=R.Options(tol=1e-8, max_al=60))
    except (np.linalg.LinAlgError, ValueError, FloatingPointError):
        return False
    return r.converged and np.abs(r.x - xc).max() <= 1e-6 * np.abs(xc).max()


def _prox_is_argmin():
    from scipy.optimize import minimize_scalar
    l1, l2, s = 0.3, 2.5, 0.7
    for x in np.linspace(-3, 3, 13):
        res = minimize_scalar(lambda t: l1 * abs(t) + 0.5 * l2 * t * t + (t - x) ** 2 / (2 * s),
                              bracket=(-50, 50), method="brent", tol=1e-14)
        if abs(R.prox_sigma_p(np.array([x]), s, l1, l2)[0] - res.x) > 1e-7:
            return False
    return True


def _p_star_is_conjugate():
    from scipy.optimize import minimize_scalar
    l1, l2 = 0.3, 2.5
    for z in [-2.0, -0.1, 0.5, 1.7]:
        res = minimize_scalar(lambda x: -(z * x - l1 * abs(x) - 0.5 * l2 * x * x), bounds=(-1e3, 1e3),
                              method="bounded", options={"xatol": 1e-12})
        if abs(R.p_star(np.array([z]), l1, l2) + res.fun) > 1e-8:
            return False
    return True


def _smw_ok():
    rng = np.random.default_rng(0)
    AJt = rng.normal(size=(7, 20))
    g = rng.normal(size=20)
    d = R.newton_direction(AJt, g, 0.37)
    return np.allclose((np.eye(20) + 0.37 * AJt.T @ AJt) @ d, -g, atol=1e-10)


def _grad_fd_ok():
    p = synth.make_problem(12, 30, k=3, seed=2)
    l1, l2 = R.lambdas(p.At, p.b, 0.7, 0.4)
    rng = np.random.default_rng(1)
    x, y, s = rng.normal(size=30) * 0.1, rng.normal(size=12), 0.5
    g = R.grad_psi(y, x, p.At, p.b, s, l1, l2)
    h = 1e-6
    fd = np.array([(R.psi(y + h * e, x, p.At, p.b, s, l1, l2) - R.psi(y - h * e, x, p.At, p.b, s, l1, l2)) / (2 * h)
                   for e in np.eye(12)])
    return np.allclose(g, fd, rtol=1e-5, atol=1e-6 * np.abs(g).max())


def test_unmutated_pins_pass():
    assert _solution_matches_cd() and _prox_is_argmin() and _p_star_is_conjugate() and _smw_ok() and _grad_fd_ok()


def test_mutant_prox_without_l2_scaling(monkeypatch):
    orig = R.prox_sigma_p
    monkeypatch.setattr(R, "prox_sigma_p", lambda t, s, l1, l2: orig(t, s, l1, l2) * (1 + s * l2))
    assert not _prox_is_argmin()
    assert not _solution_matches_cd()


def test_mutant_prox_wrong_threshold(monkeypatch):
    orig = R.prox_sigma_p
    monkeypatch.setattr(R, "prox_sigma_p", lambda t, s, l1, l2: orig(t, 1.0, l1, l2) * (1 + l2) / (1 + s * l2))
    assert not _prox_is_argmin()


def test_mutant_p_star_missing_half(monkeypatch):
    orig = R.p_star
    monkeypatch.setattr(R, "p_star", lambda z, l1, l2: 2.0 * orig(z, l1, l2))
    assert not _p_star_is_conjugate()


def test_mutant_h_star_sign(monkeypatch):
    # psi only steers the line search, so the final solution can survive this mistake;
    # the finite-difference pin of eq. grad_phy against psi catches it.
    monkeypatch.setattr(R, "h_star", lambda y, b: 0.5 * (y @ y) - b @ y)
    assert not _grad_fd_ok()


def test_mutant_smw_kappa_not_inverted(monkeypatch):
    def bad(AJt, g, kappa):
        r, m = AJt.shape
        if r == 0:
            return -g.copy()
        G = np.eye(r) * kappa + AJt @ AJt.T
        q = sla.cho_solve(sla.cho_factor(G, lower=True), AJt @ g)
        return -(g - AJt.T @ q)
    monkeypatch.setattr(R, "newton_direction", bad)
    assert not _smw_ok()


def test_mutant_smw_transposed_operand(monkeypatch):
    def bad(AJt, g, kappa):
        r, m = AJt.shape
        G = np.eye(r) / kappa + AJt @ AJt.T
        q = sla.cho_solve(sla.cho_factor(G, lower=True), AJt @ g)
        return -(g + AJt.T @ q)
    monkeypatch.setattr(R, "newton_direction", bad)
    assert not _smw_ok()


def test_mutant_active_set_threshold(monkeypatch):
    monkeypatch.setattr(R, "active_set", lambda v, s, l1: np.flatnonzero(np.abs(v) > l1))
    assert not _solution_matches_cd()


def _null_model_at_lambda_max():
    # lam_max (Sec. 4.1) is the smallest penalty whose solution is the null model: at
    # c = 1 the solution must be x = 0 (and then y = -b)
    p = synth.make_problem(30, 120, k=4, seed=8)
    l1, l2 = R.lambdas(p.At, p.b, 0.6, 1.0)
    r = R.solve(p.At, p.b, l1, l2)
    return r.converged and np.all(r.x == 0.0)


def _psi_is_lagrangian_at_z_bar():
    # Prop. 2: psi(y) = L_sigma(y, z_bar(y) | x)
    p = synth.make_problem(20, 60, k=4, seed=9)
    l1, l2 = R.lambdas(p.At, p.b, 0.7, 0.4)
    rng = np.random.default_rng(3)
    x, y, s = rng.normal(size=60) * (rng.random(60) < 0.3), rng.normal(size=20), 0.6
    z = R.z_bar(y, x, p.At, s, l1, l2)
    return np.isclose(R.psi(y, x, p.At, p.b, s, l1, l2), R.aug_lagrangian(y, z, x, p.At, p.b, s, l1, l2), rtol=1e-12)


def _mxm_branch_ok():
    # r >= m takes the m x m system; V = I + kappa A_J A_J^T is pinned by finite
    # differences of grad psi (test_oracle_psi.py)
    rng = np.random.default_rng(4)
    AJt = rng.normal(size=(26, 20))
    g = rng.normal(size=20)
    d = R.newton_direction(AJt, g, 0.37)
    return np.allclose((np.eye(20) + 0.37 * AJt.T @ AJt) @ d, -g, atol=1e-10)


def test_unmutated_extra_pins_pass():
    assert _null_model_at_lambda_max() and _psi_is_lagrangian_at_z_bar() and _mxm_branch_ok()


def test_mutant_lambdas_alpha_swapped(monkeypatch):
    def bad(At, b, alpha, c):
        g = np.abs(np.asarray(At) @ np.asarray(b)).max()
        return (1.0 - alpha) / alpha * c * g, c * g
    monkeypatch.setattr(R, "lambdas", bad)
    assert not _null_model_at_lambda_max()


def test_mutant_z_bar_without_sigma(monkeypatch):
    monkeypatch.setattr(R, "z_bar", lambda y, x, At, s, l1, l2: R.prox_p_star_over_sigma(x - s * (At @ y), 1.0, l1, l2))
    assert not _psi_is_lagrangian_at_z_bar()


def test_mutant_mxm_branch_without_kappa(monkeypatch):
    orig = R.newton_direction

    def bad(AJt, g, kappa):
        r, m = AJt.shape
        if r < m:
            return orig(AJt, g, kappa)
        M = np.eye(m) + AJt.T @ AJt
        return -sla.cho_solve(sla.cho_factor(M, lower=True), g)
    monkeypatch.setattr(R, "newton_direction", bad)
    assert not _mxm_branch_ok()


def _cg_within_krylov_bound():
    # V = I + kappa A_J A_J^T has rank(A_J) + 1 distinct eigenvalues: CG needs at most that many steps
    rng = np.random.default_rng(5)
    AJt, g = rng.normal(size=(3, 200)), rng.normal(size=200)
    d, it = R.newton_direction_cg(AJt, g, 0.05, rtol=1e-12)
    V = np.eye(200) + 0.05 * AJt.T @ AJt
    return it <= 5 and np.linalg.norm(V @ d + g) <= 1e-11 * np.linalg.norm(g)


def _cg_mutant(alpha_fn=None, beta_zero=False):
    def cg(AJt, g, kappa, rtol=1e-10, maxiter=None, history=None):
        m = g.size
        d, res = np.zeros(m), -g.copy()
        p, rr = res.copy(), res @ res
        it = 0
        while np.sqrt(rr) > rtol * np.linalg.norm(g) and it < (10 * m if maxiter is None else maxiter):
            Vp = p + kappa * (AJt.T @ (AJt @ p))
            alpha = alpha_fn(rr, p, Vp) if alpha_fn else rr / (p @ Vp)
            d, res = d + alpha * p, res - alpha * Vp
            rr_next = res @ res
            p = res + (0.0 if beta_zero else rr_next / rr) * p
            rr, it = rr_next, it + 1
        return d, it
    return cg


def test_unmutated_cg_pin_passes():
    assert _cg_within_krylov_bound()


def test_mutant_cg_step_without_V(monkeypatch):
    monkeypatch.setattr(R, "newton_direction_cg", _cg_mutant(alpha_fn=lambda rr, p, Vp: rr / (p @ p)))
    assert not _cg_within_krylov_bound()


def test_mutant_cg_without_conjugation(monkeypatch):
    monkeypatch.setattr(R, "newton_direction_cg", _cg_mutant(beta_zero=True))
    assert not _cg_within_krylov_bound()
