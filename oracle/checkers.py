"""Independent solution checkers that pin the SsNAL-EN oracle (test infrastructure only).

None of these uses the dual, the augmented Lagrangian or the Newton system;
they characterise the Elastic Net minimiser of the objective (Sec. 1)
directly.  For lam2 > 0 the objective is strongly convex, so the minimiser
is unique and every checker must agree with SsNAL-EN on it.
"""
from __future__ import annotations

import itertools

import numpy as np


def soft(t, tau):
    """Soft-thresholding: sign(t) max(|t| - tau, 0) (eq. prox_l1)."""
    return np.sign(t) * np.maximum(np.abs(t) - tau, 0.0)


def primal_objective(At, b, x, lam1, lam2):
    """P(x) = 1/2 ||A x - b||^2 + lam1 ||x||_1 + lam2/2 ||x||^2 (Sec. 1)."""
    r = np.asarray(At, dtype=np.float64).T @ x - b
    return 0.5 * (r @ r) + lam1 * np.abs(x).sum() + 0.5 * lam2 * (x @ x)


def dual_objective(At, b, y, lam1, lam2):
    """D(y) = -h*(y) - p*(-A^T y) for lam2 > 0 (every y is dual feasible with
    z = -A^T y, since p* of Prop. 1 is finite everywhere).  Weak duality gives
    P(x) >= D(y); equality holds at the optimum."""
    u = np.asarray(At, dtype=np.float64) @ y
    ps = (np.maximum(np.abs(u) - lam1, 0.0) ** 2).sum() / (2.0 * lam2)
    return -(0.5 * (y @ y) + b @ y) - ps


def kkt_violation(At, b, x, lam1, lam2):
    """Max violation of the Elastic Net optimality conditions
    a_j^T (b - A x) - lam2 x_j in lam1 * d|x_j|  (subgradient of the objective),
    relative to 1 + lam1."""
    At = np.asarray(At, dtype=np.float64)
    c = At @ (b - At.T @ x) - lam2 * x
    on = x != 0
    viol_on = np.abs(c[on] - lam1 * np.sign(x[on]))
    viol_off = np.maximum(np.abs(c[~on]) - lam1, 0.0)
    v = max(viol_on.max(initial=0.0), viol_off.max(initial=0.0))
    return v / (1.0 + lam1)


def brute_force(At, b, lam1, lam2):
    """Exhaustive sign-pattern enumeration, n <= 10.

    For every pattern s in {-1,0,1}^n with support S solve the stationarity
    equations (A_S^T A_S + lam2 I) x_S = A_S^T b - lam1 s_S; accept the pattern
    whose solution has exactly the signs s_S and whose off-support correlations
    satisfy |a_j^T (b - A x)| <= lam1.  Returns the unique accepted x.
    """
    At = np.asarray(At, dtype=np.float64)
    n = At.shape[0]
    if n > 10:
        raise ValueError("brute force is for n <= 10")
    found = []
    for pattern in itertools.product((-1, 0, 1), repeat=n):
        s = np.array(pattern, dtype=np.float64)
        S = np.flatnonzero(s)
        x = np.zeros(n)
        if len(S):
            AS = At[S]
            x[S] = np.linalg.solve(AS @ AS.T + lam2 * np.eye(len(S)), AS @ b - lam1 * s[S])
            if np.any(np.sign(x[S]) != s[S]):
                continue
        res = b - At.T @ x
        off = np.setdiff1d(np.arange(n), S)
        if np.all(np.abs(At[off] @ res) <= lam1 * (1 + 1e-12) + 1e-12):
            found.append(x)
    if len(found) != 1:
        raise RuntimeError(f"brute force found {len(found)} solutions")
    return found[0]


def coordinate_descent(At, b, lam1, lam2, tol=1e-14, max_sweeps=100_000, x0=None):
    """Cyclic coordinate descent: x_j <- soft(a_j^T r_j, lam1) / (||a_j||^2 + lam2),
    r_j = b - A x + a_j x_j, until the largest coordinate change is below
    tol * (1 + ||x||_inf).  A textbook algorithm independent of SsNAL-EN.
    """
    At = np.asarray(At, dtype=np.float64)
    n, m = At.shape
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    res = b - At.T @ x
    nrm = np.einsum("ij,ij->i", At, At)
    active = np.arange(n)
    full = True
    for _ in range(max_sweeps):
        delta = 0.0
        for j in (range(n) if full else active):
            aj = At[j]
            old = x[j]
            rho = aj @ res + nrm[j] * old
            new = soft(rho, lam1) / (nrm[j] + lam2)
            if new != old:
                res -= aj * (new - old)
                x[j] = new
                delta = max(delta, abs(new - old))
        scale = 1.0 + np.abs(x).max()
        if delta <= tol * scale:
            if full:
                return x
            full = True           # confirm with a full sweep
        else:
            if full:
                active = np.flatnonzero(x)
            full = False
    raise RuntimeError("coordinate descent did not converge")


def orthogonal_closed_form(At, b, lam1, lam2):
    """For mutually orthogonal columns with norms nu_j the objective separates:
    x_j = soft(a_j^T b, lam1) / (nu_j^2 + lam2); orthonormal columns give
    soft(A^T b, lam1) / (1 + lam2)."""
    At = np.asarray(At, dtype=np.float64)
    nu2 = np.einsum("ij,ij->i", At, At)
    return soft(At @ b, lam1) / (nu2 + lam2)


def ridge_closed_form(At, b, lam2):
    """lam1 = 0: x = A^T (A A^T + lam2 I)^{-1} b (the ridge solution)."""
    At = np.asarray(At, dtype=np.float64)
    m = At.shape[1]
    return At @ np.linalg.solve(At.T @ At + lam2 * np.eye(m), b)
