"""SsNAL-EN in plain FP64 NumPy (oracle; test infrastructure only).

Problem (Sec. 1, objective eq.):  min_x 1/2 ||A x - b||^2 + lam1 ||x||_1 + lam2/2 ||x||^2,
A is m x n (n >> m).  Storage here: ``At`` (n, m) with At[j] = column j of A.

The method (Sec. 3, Algorithm 1) is an augmented Lagrangian (AL) method on the
dual (D): min_{y,z} h*(y) + p*(z) s.t. A^T y + z = 0, whose inner sub-problem is
solved by a semi-smooth Newton (SsN) method on psi(y) (Prop. 2).

Readings of points the paper leaves open (the CUDA path takes the same readings; the
conjugate-gradient branch below applies only where the device supports CG solves):
  * grad h*(y) = y + b  (Sec. 3 writes "y - b" once, "y + b" twice; h*(y) = 1/2||y||^2 + b^T y).
  * x^0 = 0 or the warm start, y^0 = A x^0 - b, sigma^0 = 5e-3 grown x5 per AL
    iteration and capped at sigma_max (Sec. 4.1; Algorithm 1 step (2)).
  * SsN stop: ||grad psi(y)|| / (1 + ||b||) <= tol, i.e. res(kkt1) at the tentative
    x = prox_{sigma p}(x - sigma A^T y); AL stop: res(kkt1) <= tol and res(kkt3) <= tol.
  * Line search: s in {1, beta, beta^2, ...}, beta = 1/2, mu = 0.2, at most max_ls
    trials; if none passes, the last trial step is taken.
  * The active set uses the strict test |v_j| > sigma lam1 (eq. for Q).
  * SMW form iff 0 < r < m; m x m form iff r >= m; r = 0 gives d = -grad psi.
  * Conjugate gradients replace the direct Newton solve when m and r both exceed 1e4
    (Sec. 3.2), started at d = 0 and stopped at ||V d + g|| <= 1e-10 ||g|| (the paper
    gives no CG tolerance).
  * The x update: x <- x - sigma (A^T y + z) with z from Prop. 2 (2); by the Moreau
    decomposition (Sec. 2.2) this is prox_{sigma p}(x - sigma A^T y), which is
    evaluated in that form so that inactive coordinates are exactly zero.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import scipy.linalg as sla


# --------------------------------------------------------------------------- Sec. 2
def penalty(x, lam1, lam2):
    """p(x) = lam1 ||x||_1 + lam2/2 ||x||^2 (Elastic Net penalty, Sec. 1)."""
    return lam1 * np.abs(x).sum() + 0.5 * lam2 * (x @ x)


def p_star(z, lam1, lam2):
    """Conjugate of the Elastic Net penalty, Prop. 1 (eq. p_star).

    p*(z) = 1/(2 lam2) sum_i { (z_i - lam1)^2 if z_i >= lam1; 0 if |z_i| < lam1;
                              (z_i + lam1)^2 if z_i <= -lam1 }.
    """
    z = np.asarray(z, dtype=np.float64)
    out = np.where(z >= lam1, (z - lam1) ** 2, np.where(z <= -lam1, (z + lam1) ** 2, 0.0))
    return out.sum() / (2.0 * lam2)


def h_star(y, b):
    """h*(y) = 1/2 ||y||^2 + b^T y for h(u) = 1/2 ||u - b||^2 (Sec. 3)."""
    return 0.5 * (y @ y) + b @ y


def prox_sigma_p(t, sigma, lam1, lam2):
    """prox_{sigma p}(t), componentwise (eq. prox_elastic, left):

    1/(1 + sigma lam2) * { t - sigma lam1 if t >= sigma lam1; 0 if |t| < sigma lam1;
                           t + sigma lam1 if t <= -sigma lam1 }.
    """
    t = np.asarray(t, dtype=np.float64)
    thr = sigma * lam1
    out = np.where(t >= thr, t - thr, np.where(t <= -thr, t + thr, 0.0))
    return out / (1.0 + sigma * lam2)


def prox_p_star_over_sigma(t, sigma, lam1, lam2):
    """prox_{p*/sigma}(t / sigma), componentwise (eq. prox_elastic, right):

    { (t lam2 + lam1)/(1 + sigma lam2) if t >= sigma lam1; t/sigma if |t| < sigma lam1;
      (t lam2 - lam1)/(1 + sigma lam2) if t <= -sigma lam1 }.
    """
    t = np.asarray(t, dtype=np.float64)
    thr = sigma * lam1
    den = 1.0 + sigma * lam2
    return np.where(t >= thr, (t * lam2 + lam1) / den,
                    np.where(t <= -thr, (t * lam2 - lam1) / den, t / sigma))


# --------------------------------------------------------------------------- Sec. 3
def aug_lagrangian(y, z, x, At, b, sigma, lam1, lam2):
    """L_sigma(y, z, x) = h*(y) + p*(z) - x^T(A^T y + z) + sigma/2 ||A^T y + z||^2 (eq. lagrangian)."""
    r = At @ y + z
    return h_star(y, b) + p_star(z, lam1, lam2) - x @ r + 0.5 * sigma * (r @ r)


def psi(y, x, At, b, sigma, lam1, lam2):
    """psi(y) of Prop. 2 (1):
    h*(y) + (1 + sigma lam2)/(2 sigma) ||prox_{sigma p}(x - sigma A^T y)||^2 - ||x||^2/(2 sigma).
    """
    w = prox_sigma_p(x - sigma * (At @ y), sigma, lam1, lam2)
    return h_star(y, b) + (1.0 + sigma * lam2) / (2.0 * sigma) * (w @ w) - (x @ x) / (2.0 * sigma)


def z_bar(y, x, At, sigma, lam1, lam2):
    """z-bar = prox_{p*/sigma}(x/sigma - A^T y) (Prop. 2 (2)); the argument of the
    componentwise formula is t = x - sigma A^T y, i.e. prox_{p*/sigma}(t / sigma)."""
    return prox_p_star_over_sigma(x - sigma * (At @ y), sigma, lam1, lam2)


def grad_psi(y, x, At, b, sigma, lam1, lam2):
    """grad psi(y) = y + b - A prox_{sigma p}(x - sigma A^T y) (eq. grad_phy)."""
    w = prox_sigma_p(x - sigma * (At @ y), sigma, lam1, lam2)
    J = np.flatnonzero(w)
    return y + b - At[J].T @ w[J]


def active_set(v, sigma, lam1):
    """J = { j : |v_j| > sigma lam1 } (eq. Q_def), sorted ascending."""
    return np.flatnonzero(np.abs(v) > sigma * lam1)


def newton_direction(AJt, g, kappa):
    """Solve (I_m + kappa A_J A_J^T) d = -g (eq. AJ_system).

    r = 0: d = -g.  0 < r < m: Sherman-Morrison-Woodbury (eq. smw_formula),
    d = -(g - A_J (kappa^{-1} I_r + A_J^T A_J)^{-1} A_J^T g).  r >= m: Cholesky
    of the m x m matrix.  ``AJt`` is A_J transposed, shape (r, m).
    """
    r, m = AJt.shape
    if r == 0:
        return -g.copy()
    if r < m:
        G = np.eye(r) / kappa + AJt @ AJt.T
        q = sla.cho_solve(sla.cho_factor(G, lower=True), AJt @ g)
        return -(g - AJt.T @ q)
    M = np.eye(m) + kappa * (AJt.T @ AJt)
    return -sla.cho_solve(sla.cho_factor(M, lower=True), g)


def newton_direction_cg(AJt, g, kappa, rtol=1e-10, maxiter=None, history=None):
    """Approximate solve of (I_m + kappa A_J A_J^T) d = -g (eq. AJ_system) by conjugate
    gradients, which Algorithm 1 step (1) allows and Sec. 3.2 proposes once m and r both
    exceed 1e4.  Matrix-free: V p = p + kappa A_J (A_J^T p).  Textbook CG started at d = 0;
    it stops when ||V d + g|| <= rtol ||g|| or after maxiter iterations (default 10 m: in
    exact arithmetic at most m are needed, rounding can add some).  If
    ``history`` is a list, the iterate of every iteration is appended to it.  Returns
    (d, iterations)."""
    AJt = np.asarray(AJt, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = g.size
    d = np.zeros(m)
    res = -g.copy()  # -g - V d at d = 0
    p = res.copy()
    rr = res @ res
    stop = rtol * np.sqrt(g @ g)
    limit = 10 * m if maxiter is None else maxiter
    it = 0
    while np.sqrt(rr) > stop and it < limit:
        Vp = p + kappa * (AJt.T @ (AJt @ p))
        alpha = rr / (p @ Vp)
        d = d + alpha * p
        res = res - alpha * Vp
        rr_next = res @ res
        p = res + (rr_next / rr) * p
        rr = rr_next
        it += 1
        if history is not None:
            history.append(d.copy())
    return d, it


@dataclasses.dataclass
class Options:
    sigma0: float = 5e-3       # Sec. 4.1
    sigma_growth: float = 5.0  # Sec. 4.1
    sigma_max: float = 1e8     # Algorithm 1 step (2): sigma increases to sigma_inf
    mu: float = 0.2            # Sec. 4.1, Armijo constant in (0, 1/2)
    beta: float = 0.5          # backtracking factor (unstated in the paper)
    tol: float = 1e-6          # Sec. 4.1
    max_al: int = 100
    max_newton: int = 50
    max_ls: int = 40
    cg_above: int = 10_000     # CG Newton solve when m and r both exceed this (Sec. 3.2)
    cg_rtol: float = 1e-10


@dataclasses.dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    sigma: float
    al_iters: int
    newton_iters: int
    ls_trials: int
    kkt1: float
    kkt3: float
    converged: bool
    r_history: list
    seconds: float


def solve(At, b, lam1, lam2, x0=None, y0=None, opts: Options | None = None) -> Result:
    """SsNAL-EN, Algorithm 1, in plain FP64.

    AL loop (upper half): approximately minimise L_sigma(y, z | x) over (y, z)
    through psi (Prop. 2), update x by eq. update_x, test res(kkt3) and
    res(kkt1) (eq. kkt_res), grow sigma.  SsN loop (lower half): Newton
    direction from the generalized Hessian V = I + kappa A_J A_J^T
    (eqs. Q_def, AJ_system, smw_formula), Armijo backtracking (eq. line_search),
    y update.
    """
    opts = opts or Options()
    t0 = time.perf_counter()
    At = np.asarray(At, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n, m = At.shape
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    y = (At.T @ x - b) if y0 is None else np.array(y0, dtype=np.float64)
    nb1 = 1.0 + np.linalg.norm(b)
    sigma = opts.sigma0
    newton = ls_total = 0
    r_hist = []
    kkt1 = kkt3 = np.inf
    z = np.zeros(n)
    it = 0
    converged = False
    for it in range(1, opts.max_al + 1):
        # ---- SsN on psi(y) for the current x, sigma (Algorithm 1, lower half)
        for _ in range(opts.max_newton):
            u = At @ y                                   # A^T y, fresh every step
            v = x - sigma * u
            J = active_set(v, sigma, lam1)               # eq. Q_def
            w = prox_sigma_p(v, sigma, lam1, lam2)       # eq. prox_elastic
            g = y + b - At[J].T @ w[J]                   # eq. grad_phy
            if np.linalg.norm(g) / nb1 <= opts.tol:
                break
            kappa = sigma / (1.0 + sigma * lam2)
            if m > opts.cg_above and len(J) > opts.cg_above:
                d, _ = newton_direction_cg(At[J], g, kappa, opts.cg_rtol)   # Sec. 3.2
            else:
                d = newton_direction(At[J], g, kappa)    # eqs. AJ_system / smw_formula
            r_hist.append(len(J))
            newton += 1
            psi0 = psi(y, x, At, b, sigma, lam1, lam2)
            gd = g @ d
            s = 1.0
            for trial in range(opts.max_ls):             # eq. line_search
                ls_total += 1
                if psi(y + s * d, x, At, b, sigma, lam1, lam2) <= psi0 + opts.mu * s * gd:
                    break
                if trial < opts.max_ls - 1:
                    s *= opts.beta
            y = y + s * d
        # ---- multiplier update (Algorithm 1, upper half, step (2))
        u = At @ y
        z = z_bar(y, x, At, sigma, lam1, lam2)           # Prop. 2 (2)
        kkt3 = np.linalg.norm(u + z) / (1.0 + np.linalg.norm(y) + np.linalg.norm(z))
        x = prox_sigma_p(x - sigma * u, sigma, lam1, lam2)   # = x - sigma (A^T y + z), Moreau
        supp = np.flatnonzero(x)
        kkt1 = np.linalg.norm(y + b - At[supp].T @ x[supp]) / nb1
        if kkt1 <= opts.tol and kkt3 <= opts.tol:
            converged = True
            break
        sigma = min(sigma * opts.sigma_growth, opts.sigma_max)
    return Result(x=x, y=y, z=z, sigma=sigma, al_iters=it, newton_iters=newton, ls_trials=ls_total,
                  kkt1=kkt1, kkt3=kkt3, converged=converged, r_history=r_hist,
                  seconds=time.perf_counter() - t0)


def lambdas(At, b, alpha, c):
    """lam1 = alpha c lam_max, lam2 = (1 - alpha) c lam_max, lam_max = ||A^T b||_inf / alpha
    (Sec. 4.1), evaluated as lam1 = c ||A^T b||_inf and lam2 = (1-alpha)/alpha c ||A^T b||_inf."""
    g = np.abs(np.asarray(At, dtype=np.float64) @ np.asarray(b, dtype=np.float64)).max()
    return c * g, (1.0 - alpha) / alpha * c * g


def path(At, b, alpha, c_grid, max_active=0, opts: Options | None = None):
    """Warm-started regularization path (Sec. 3.3).

    Grid points are visited in the given (descending) order; each fit starts
    from the previous solution x (and y^0 = A x^0 - b); sigma restarts at
    sigma0 at every point.  With ``max_active`` > 0 the path stops after the
    first point whose solution has at least that many nonzeros.
    """
    At = np.asarray(At, dtype=np.float64)
    g = np.abs(At @ b).max()
    x = np.zeros(At.shape[0])
    out = []
    for c in c_grid:
        lam1 = c * g
        lam2 = (1.0 - alpha) / alpha * c * g
        res = solve(At, b, lam1, lam2, x0=x, opts=opts)
        res.lam1, res.lam2, res.c = lam1, lam2, c
        out.append(res)
        x = res.x
        if max_active and np.count_nonzero(x) >= max_active:
            break
    return out


# --------------------------------------------------------------------------- parameter tuning
def en_degrees_of_freedom(At, x, lam2):
    """Elastic Net degrees of freedom of a solution (Sec. 3.3, after eq. gcv_bic):
    nu = tr( A_J (A_J^T A_J + lam2 I_r)^{-1} A_J^T ), J the active set of x.  Written out with a
    dense solve; nu = 0 for an empty active set."""
    At = np.asarray(At, dtype=np.float64)
    J = np.flatnonzero(x)
    if J.size == 0:
        return 0.0
    AJ = At[J].T                                        # m x r
    G = AJ.T @ AJ + lam2 * np.eye(J.size)
    H = AJ @ np.linalg.solve(G, AJ.T)                   # the hat-like matrix
    return float(np.trace(H))


def debiased_rss(At, b, x):
    """Residual sum of squares after the de-biasing of Sec. 3.3: ordinary least squares on the
    active set of x, rss = || b - A_J x_ols ||^2 (lstsq; zero when the fit interpolates)."""
    At = np.asarray(At, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    J = np.flatnonzero(x)
    if J.size == 0:
        return float(b @ b)
    AJ = At[J].T
    coef, *_ = np.linalg.lstsq(AJ, b, rcond=None)
    r = b - AJ @ coef
    return float(r @ r)


def tuning_criteria(At, b, x, lam2):
    """(nu, rss, gcv, e-bic) of eq. gcv_bic for one solution:
    gcv = rss / m / (1 - nu/m)^2,  e-bic = log(rss / m) + (nu / m) (log m + log n)."""
    At = np.asarray(At, dtype=np.float64)
    n, m = At.shape
    nu = en_degrees_of_freedom(At, x, lam2)
    rss = debiased_rss(At, b, x)
    gcv = (rss / m) / (1.0 - nu / m) ** 2 if nu != m else np.inf
    ebic = np.log(rss / m) + (nu / m) * (np.log(m) + np.log(n)) if rss > 0 else -np.inf
    return nu, rss, gcv, ebic
