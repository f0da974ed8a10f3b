"""GPU parity of the FP64 Newton system (eqs. AJ_system, smw_formula) and of the fallback
to it: the Newton matrix formed, factored and solved in FP64 on the device, used when the
FP32 factor fails or its iterative refinement does not contract, or always on request
(options.newton_fp64 = 1).

The FP32 factor's relative error is about cond(G) 2^-24; duplicated columns of A make
A_J^T A_J singular, so cond(G) = 1 + kappa ||A_J||^2 and a large kappa (a large sigma
with a small lambda2, i.e. alpha close to 1) puts the FP32 solve out of reach of its
refinement.  Those cases must still match the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2006_03970_gb300 as pkg  # noqa: E402
from oracle import ssnal_en_ref as R  # noqa: E402
from paper_2006_03970_gb300 import synth  # noqa: E402

from test_gpu_parity import assert_parity, dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_03970_gb300 import build
    build.build()
    pkg.load_library()


def _newton(At, J, g, kappa, options):
    m = At.shape[1]
    r = len(J)
    ctx = pkg.Context(At, options=options)
    gd = torch.empty(m, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_grad(ctx.ctx, dev(J, torch.int32) if r else None, dev(np.zeros(r)) if r else None, r,
                         dev(-g), dev(np.zeros(m)), gd)  # gathers A_J
    d = torch.empty(m, dtype=torch.float64, device="cuda")
    st = pkg.ssnal_en_op_newton(ctx.ctx, r, kappa, dev(g), d)
    ctx.close()
    return st, d.cpu().numpy()


def _cond(AJt, kappa):
    r, m = AJt.shape
    G = np.eye(r) / kappa + AJt @ AJt.T if r < m else np.eye(m) + kappa * AJt.T @ AJt
    ev = np.linalg.eigvalsh(G)
    return ev[-1] / ev[0]


# ---------------------------------------------------------------- the FP64 system on request
@pytest.mark.parametrize("m,r", [(30, 1), (30, 29), (30, 30), (30, 31), (5, 7), (33, 64), (100, 250), (257, 65),
                                 (500, 120), (300, 200), (700, 600), (1000, 999), (900, 1500), (2100, 2200),
                                 (4096, 300)])
def test_newton_direction_fp64_system(m, r):
    rng = np.random.default_rng(3 * m + r)
    At = rng.normal(size=(r + 10, m))
    J = np.arange(r, dtype=np.int32)
    g = rng.normal(size=m)
    kappa = 0.05
    st, d = _newton(At, J, g, kappa, pkg.ssnal_en_default_options(newton_fp64=1))
    assert st == pkg.OK
    ref = R.newton_direction(At[J], g, kappa)
    np.testing.assert_allclose(d, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


# ---------------------------------------------------------------- ill-conditioned Newton matrices
@pytest.mark.parametrize("kappa", [1e2, 1e4])
@pytest.mark.parametrize("m,r,dup", [(300, 290, 0), (300, 300, 0), (300, 450, 0), (128, 96, 8), (200, 120, 20),
                                     (64, 64, 4)])
def test_newton_direction_ill_conditioned(m, r, dup, kappa):
    # default options: FP32 factor + refinement, the FP64 system when that is not accurate.
    # `dup` columns of A_J are exact copies of others (A_J^T A_J singular).
    rng = np.random.default_rng(m + r + dup)
    At = rng.normal(size=(r + 10, m))
    if dup:
        At[r - dup:r] = At[:dup]
    J = np.arange(r, dtype=np.int32)
    g = rng.normal(size=m)
    st, d = _newton(At, J, g, kappa, pkg.ssnal_en_default_options())
    assert st == pkg.OK
    ref = R.newton_direction(At[J], g, kappa)
    cond = _cond(At[J], kappa)
    err = np.abs(d - ref).max() / np.abs(ref).max()
    # the single-step entry point refines the FP32 solve until its corrections stop
    # shrinking (the accuracy of the FP64 residual), or takes the FP64 system when the
    # refinement does not contract: either way the result is accurate to a small multiple
    # of cond 2^-53
    tol = max(1e-10, 1e3 * cond * np.finfo(float).eps)
    assert err <= tol, (err, tol, cond)


# ---------------------------------------------------------------- whole fits
def _dup_problem(m, n, k, seed, ndup):
    p = synth.make_problem(m, n, k=k, seed=seed, snr=2)
    At = p.At.copy()
    supp = np.flatnonzero(p.x_true)
    for i in range(ndup):  # the last columns copy true predictors: they enter J together
        At[n - 1 - i] = At[supp[i]]
    return At, p.b


def test_fit_falls_back_to_the_fp64_system_and_matches_the_oracle():
    # lambda2 = 1e-6 (kappa < 1/lambda2 = 1e6) and sigma0 = 1e4: kappa ~ 1e4 .. 1e6 from the
    # first Newton step, and the duplicated columns make cond(G) ~ 1 + kappa ||A_J||^2, up to
    # ~3e8 along the oracle's iterates: far beyond the FP32 factor
    At, b = _dup_problem(100, 1000, 10, 5, 5)
    lam1, _ = R.lambdas(At, b, 0.999, 0.2)
    lam2 = 1e-6
    o = pkg.ssnal_en_default_options(sigma0=1e4)
    ctx = pkg.Context(At, options=o)
    x, _, res = ctx.solve(b, lam1, lam2)
    ro = R.solve(At, b, lam1, lam2, opts=R.Options(sigma0=1e4))
    ctx.close()
    assert ro.converged and res.status == pkg.OK
    assert res.newton_fp64 > 0  # the fallback ran
    assert_parity(At, b, lam1, lam2, x.cpu().numpy(), ro)


@pytest.mark.parametrize("m,n,c,seed", [(200, 2000, 0.001, 1), (120, 3000, 0.001, 3), (60, 2000, 0.01, 1)])
def test_fit_parity_alpha_0999(m, n, c, seed):
    # alpha = 0.999: lambda2 ~ 1e-3 lambda1, kappa grows with sigma up to ~1e3 and the
    # Newton matrices reach condition numbers of ~1e5-1e6 (r close to m).  The problem is
    # barely strongly convex, so the iterate where a solver stops at KKT 1e-6 can sit
    # ~1e-6 (relative) from another correct solver's: both sides run to KKT 1e-8, where
    # the solutions must agree to the 1e-6 bar whatever the rounding order.
    p = synth.make_problem(m, n, k=30 if m > 100 else 10, seed=seed, snr=2)
    lam1, lam2 = R.lambdas(p.At, p.b, 0.999, c)
    ro = R.solve(p.At, p.b, lam1, lam2, opts=R.Options(tol=1e-8))
    for forced in (0, 1):
        ctx = pkg.Context(p.At, options=pkg.ssnal_en_default_options(newton_fp64=forced, tol=1e-8))
        x, _, res = ctx.solve(p.b, lam1, lam2)
        ctx.close()
        assert ro.converged and res.status == pkg.OK, res.as_dict()
        if forced:
            assert res.newton_fp64 == res.newton_iters
        assert_parity(p.At, p.b, lam1, lam2, x.cpu().numpy(), ro)


def test_path_with_the_fp64_system_matches_the_oracle():
    p = synth.make_problem(80, 3000, k=8, seed=12, block=20, rho=0.7)
    grid = synth.path_grid(6, 0.05)
    ctx = pkg.Context(p.At, options=pkg.ssnal_en_default_options(newton_fp64=1))
    X, res, done = ctx.path(p.b, 0.6, grid)
    ro = R.path(p.At, p.b, 0.6, grid)
    assert done == len(grid)
    Xg = X.cpu().numpy()
    for k, rk in enumerate(ro):
        assert res[k].status == pkg.OK
        assert_parity(p.At, p.b, rk.lam1, rk.lam2, Xg[k], rk)
    ctx.close()


@pytest.mark.parametrize("m,r", [(300, 250), (300, 300)])
def test_newton_direction_hopeless_for_fp32_comes_from_fp64(m, r):
    # cond(G) ~ 1e9: the FP32 solve has no correct digit, the FP64 system has about seven
    rng = np.random.default_rng(m * r)
    At = rng.normal(size=(r + 10, m))
    At[r - 20:r] = At[:20]  # duplicated columns: A_J^T A_J singular
    J = np.arange(r, dtype=np.int32)
    g = rng.normal(size=m)
    kappa = 1e6
    cond = _cond(At[J], kappa)
    assert cond * 2.0 ** -24 >= 1.0
    st, d = _newton(At, J, g, kappa, pkg.ssnal_en_default_options())
    assert st == pkg.OK
    ref = R.newton_direction(At[J], g, kappa)
    err = np.abs(d - ref).max() / np.abs(ref).max()
    assert err <= max(1e-10, 1e3 * cond * np.finfo(float).eps), (err, cond)
