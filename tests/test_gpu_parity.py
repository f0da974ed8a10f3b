"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Bars (from the problem statement of the FP64 path):
  * relative objective gap |P(x_gpu) - P(x_or)| / max(1, |P(x_or)|) <= 1e-9,
  * ||x_gpu - x_or||_inf / ||x_or||_inf <= 1e-6 (x_gpu = 0 exactly when x_or = 0),
  * supports identical at every index whose final |v_j| - sigma*lam1 lies outside
    a 1e-8 relative margin (ties there are equally valid Clarke elements).
Kernel-level tests use FP64 rounding bounds derived from the arithmetic.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2006_03970_gb300 as pkg  # noqa: E402
from oracle import checkers as C  # noqa: E402
from oracle import ssnal_en_ref as R  # noqa: E402
from paper_2006_03970_gb300 import synth  # noqa: E402

OBJ_TOL = 1e-9
X_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_03970_gb300 import build
    build.build()
    pkg.load_library()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def assert_parity(At, b, lam1, lam2, x_gpu, ro, obj_tol=OBJ_TOL, x_tol=X_TOL):
    P_or = C.primal_objective(At, b, ro.x, lam1, lam2)
    P_gpu = C.primal_objective(At, b, x_gpu, lam1, lam2)
    assert abs(P_gpu - P_or) <= obj_tol * max(1.0, abs(P_or)), (P_gpu, P_or)
    xmax = np.abs(ro.x).max()
    if xmax == 0:
        assert np.all(x_gpu == 0.0)
    else:
        assert np.abs(x_gpu - ro.x).max() <= x_tol * xmax, np.abs(x_gpu - ro.x).max() / xmax
    # supports agree outside the tie margin: |x_j| = (|v_j| - sigma lam1)/(1 + sigma lam2), so an
    # entry that is nonzero on one side only must sit within the margin of the threshold
    big = np.abs(ro.x) > 1e-8 * max(xmax, 1e-300)
    assert np.all(x_gpu[big] != 0.0)
    extra = (x_gpu != 0.0) & (ro.x == 0.0)
    assert np.all(np.abs(x_gpu[extra]) <= 1e-8 * max(xmax, 1e-300))


# ---------------------------------------------------------------- a1: u = A^T y
@pytest.mark.parametrize("m,n", [(1, 1), (7, 33), (31, 1000), (100, 2000), (513, 4097), (1000, 3), (2000, 777)])
def test_at_y_stream(m, n):
    rng = np.random.default_rng(m * 7 + n)
    At = rng.normal(size=(n, m))
    y = rng.normal(size=m)
    ctx = pkg.Context(At)
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(y), u)
    ref = At @ y
    # float-float products carry 47 significant bits; the low word accumulates m roundings of 2^-24
    # relative to itself (itself ~2^-24 of the terms): |err| <= (2^-45 + m 2^-47) sum |a||y|.
    bound = (2.0 ** -45 + m * 2.0 ** -47) * (np.abs(At) @ np.abs(y)) + 1e-300
    assert np.all(np.abs(u.cpu().numpy() - ref) <= bound)
    # float-float with on-the-fly splitting (precision = 3) meets the same bound
    ctx.set_options(pkg.ssnal_en_default_options(precision=3))
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(y), u)
    assert np.all(np.abs(u.cpu().numpy() - ref) <= bound)
    # the FP64-FMA stream (precision = 2) stays within the FP64 dot-product bound
    ctx.set_options(pkg.ssnal_en_default_options(precision=2))
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(y), u)
    bound = 4 * m * np.finfo(float).eps * (np.abs(At) @ np.abs(y)) + 1e-300
    assert np.all(np.abs(u.cpu().numpy() - ref) <= bound)
    ctx.close()


@pytest.mark.parametrize("scale", [1e-200, 1e120])
def test_at_y_out_of_range_entries_use_fp64_stream(scale):
    rng = np.random.default_rng(3)
    m, n = 50, 700
    At = rng.normal(size=(n, m))
    At[17, 3] = scale  # outside [2^-100, 2^100]: the float-float split is not used
    y = rng.normal(size=m)
    ctx = pkg.Context(At)
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(y), u)
    ref = At @ y
    bound = 4 * m * np.finfo(float).eps * (np.abs(At) @ np.abs(y)) + 1e-300
    assert np.all(np.abs(u.cpu().numpy() - ref) <= bound)
    ctx.close()


@pytest.mark.parametrize("m", [2, 64, 641, 1280, 1281, 4096])
def test_at_y_stream_tile_shapes(m):
    # single-chunk tiles (several columns per warp) and row-chunked tall columns
    n = 1031
    rng = np.random.default_rng(m)
    At = rng.normal(size=(n, m))
    y = rng.normal(size=m) * 1e-3
    ctx = pkg.Context(At)
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(y), u)
    ref = At @ y
    bound = (2.0 ** -45 + m * 2.0 ** -47) * (np.abs(At) @ np.abs(y)) + 1e-300
    assert np.all(np.abs(u.cpu().numpy() - ref) <= bound)
    ctx.set_options(pkg.ssnal_en_default_options(precision=3))
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(y), u)
    assert np.all(np.abs(u.cpu().numpy() - ref) <= bound)
    ctx.close()


def test_at_y_ignores_padding_rows():
    rng = np.random.default_rng(5)
    m, n = 5, 40
    At = rng.normal(size=(n, m))
    A, _ = pkg.device_matrix(At)
    A[:, m:] = float("nan")  # lda = 6: one padding row holding NaN
    ctx = pkg.Context(A, m=m)
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(rng.normal(size=m)), u)
    assert torch.isfinite(u).all()
    ctx.close()


# ---------------------------------------------------------------- a2: prox + J
# 400_000: more entries per block than threads (several tiles of the compaction per block)
@pytest.mark.parametrize("n", [1, 255, 256, 257, 5000, 100_003, 400_000])
def test_prox_active_set(n):
    rng = np.random.default_rng(n)
    m = 8
    ctx = pkg.Context(rng.normal(size=(n, m)))
    x = rng.normal(size=n) * (rng.random(n) < 0.3)
    u = rng.normal(size=n) * 3
    sigma, l1, l2 = 0.37, 2.1, 0.8
    J = torch.empty(n, dtype=torch.int32, device="cuda")
    wJ = torch.empty(n, dtype=torch.float64, device="cuda")
    r = pkg.ssnal_en_op_prox_active(ctx.ctx, dev(x), dev(u), sigma, l1, l2, J, wJ)
    v = x - sigma * u
    Jo = R.active_set(v, sigma, l1)
    wo = R.prox_sigma_p(v, sigma, l1, l2)[Jo]
    assert r == len(Jo)
    np.testing.assert_array_equal(J[:r].cpu().numpy(), Jo)  # bit-exact indices, ascending
    np.testing.assert_array_equal(wJ[:r].cpu().numpy(), wo)  # same rounding sequence as the definition
    ctx.close()


def test_prox_active_set_ties_are_excluded():
    # |v| == sigma*lam1 exactly is not active (strict test of eq. Q_def)
    n, m = 64, 4
    ctx = pkg.Context(np.ones((n, m)))
    sigma, l1 = 0.5, 2.0
    u = np.zeros(n)
    x = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)  # |v| = 1 = sigma*lam1
    x[5] = 1.5
    J = torch.empty(n, dtype=torch.int32, device="cuda")
    wJ = torch.empty(n, dtype=torch.float64, device="cuda")
    r = pkg.ssnal_en_op_prox_active(ctx.ctx, dev(x), dev(u), sigma, l1, 0.3, J, wJ)
    assert r == 1 and J[0].item() == 5
    ctx.close()


# ---------------------------------------------------------------- a3 + a4: gather + gradient
@pytest.mark.parametrize("m,n,r", [(9, 50, 0), (9, 50, 1), (100, 2000, 37), (513, 3000, 700)])
def test_grad_gather(m, n, r):
    rng = np.random.default_rng(r + m)
    At = rng.normal(size=(n, m))
    ctx = pkg.Context(At)
    J = np.sort(rng.choice(n, size=r, replace=False)).astype(np.int32)
    wJ = rng.normal(size=r)
    y, b = rng.normal(size=m), rng.normal(size=m)
    g = torch.empty(m, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_grad(ctx.ctx, dev(J, torch.int32) if r else None, dev(wJ) if r else None, r, dev(y), dev(b), g)
    ref = y + b - At[J].T @ wJ
    bound = 4 * (r + 2) * np.finfo(float).eps * (np.abs(y) + np.abs(b) + np.abs(At[J]).T @ np.abs(wJ))
    assert np.all(np.abs(g.cpu().numpy() - ref) <= bound + 1e-300)
    ctx.close()


# ---------------------------------------------------------------- a5 + a6: Newton system
@pytest.mark.parametrize("syrk_tc", [1, 0])
@pytest.mark.parametrize("m,r", [(30, 0), (30, 1), (30, 29), (30, 30), (30, 31), (5, 7), (40, 32), (32, 40), (100, 250), (257, 65),
                                 (500, 120), (128, 129), (129, 300), (300, 200), (200, 400), (700, 600),
                                 (720, 680), (900, 800), (760, 800), (1000, 999),
                                 (1500, 1400)])
def test_newton_direction(m, r, syrk_tc):
    # syrk_tc = 1: Newton matrix on the tensor cores (three-way BF16 split, FP32 accumulation);
    # 0: FP32 FMA.  Both feed an FP32 factor refined through the FP64 panel.
    rng = np.random.default_rng(m + r)
    n = max(r, 1) + 10
    At = rng.normal(size=(n, m))
    # two refinement steps: FP32 factor error (cond * 2^-24) squared twice is below 1e-10
    ctx = pkg.Context(At, options=pkg.ssnal_en_default_options(refine_steps=2, syrk_tc=syrk_tc))
    J = np.arange(r, dtype=np.int32)
    g = rng.normal(size=m)
    gd = torch.empty(m, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_grad(ctx.ctx, dev(J, torch.int32) if r else None, dev(np.zeros(r)) if r else None, r,
                         dev(-g), dev(np.zeros(m)), gd)  # gathers A_J; gd = -g
    kappa = 0.05
    d = torch.empty(m, dtype=torch.float64, device="cuda")
    st = pkg.ssnal_en_op_newton(ctx.ctx, r, kappa, dev(g), d)
    assert st == pkg.OK
    ref = R.newton_direction(At[J], g, kappa)
    np.testing.assert_allclose(d.cpu().numpy(), ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    # the default single refinement step: error about (cond * 2^-24)^2
    ctx.set_options(pkg.ssnal_en_default_options(syrk_tc=syrk_tc))
    pkg.ssnal_en_op_newton(ctx.ctx, r, kappa, dev(g), d)
    np.testing.assert_allclose(d.cpu().numpy(), ref, rtol=1e-7, atol=1e-7 * np.abs(ref).max())
    ctx.close()


# ---------------------------------------------------------------- whole fit
def _solve_both(p, lam1, lam2, options=None):
    ctx = pkg.Context(p.At, options=options)
    x, y, res = ctx.solve(p.b, lam1, lam2)
    torch.cuda.synchronize()
    ro = R.solve(p.At, p.b, lam1, lam2)
    ctx.close()
    return x.cpu().numpy(), y.cpu().numpy(), res, ro


def test_config1_parity():
    p = synth.config1()
    lam1, lam2 = R.lambdas(p.At, p.b, p.alpha, p.c)
    xg, yg, res, ro = _solve_both(p, lam1, lam2)
    assert res.status == pkg.OK and ro.converged
    assert res.kkt1 <= 1e-6 and res.kkt3 <= 1e-6
    assert_parity(p.At, p.b, lam1, lam2, xg, ro)
    # the iteration path follows the oracle's
    assert res.al_iters == ro.al_iters
    assert abs(res.newton_iters - ro.newton_iters) <= 1
    assert res.active == np.count_nonzero(ro.x)
    P = C.primal_objective(p.At, p.b, xg, lam1, lam2)
    assert res.primal_obj == pytest.approx(P, rel=1e-12)
    assert 0 <= res.dual_gap <= 1e-6 * P


@pytest.mark.parametrize("m,n,alpha,c,seed,block,rho", [
    (40, 300, 0.8, 0.3, 1, 1, 0.0), (64, 1025, 0.5, 0.1, 2, 10, 0.7), (120, 5000, 0.95, 0.2, 3, 50, 0.5),
    (7, 500, 0.6, 0.5, 4, 1, 0.0), (300, 257, 0.7, 0.05, 5, 1, 0.0), (200, 20000, 0.9, 0.6, 6, 100, 0.7)])
def test_fit_parity(m, n, alpha, c, seed, block, rho):
    p = synth.make_problem(m, n, k=max(3, m // 20), seed=seed, block=block, rho=rho, alpha=alpha)
    lam1, lam2 = R.lambdas(p.At, p.b, alpha, c)
    xg, yg, res, ro = _solve_both(p, lam1, lam2)
    assert res.status == pkg.OK and ro.converged
    assert_parity(p.At, p.b, lam1, lam2, xg, ro)


def _golden():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "tiny_en.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_golden_tiny_gpu(case):
    At = np.ascontiguousarray(np.array(case["A"]).T)
    b = np.array(case["b"])
    o = pkg.ssnal_en_default_options(tol=1e-9)
    ctx = pkg.Context(At, options=o)
    x, _, res = ctx.solve(b, case["lam1"], case["lam2"])
    xg = x.cpu().numpy()
    assert res.status == pkg.OK
    np.testing.assert_allclose(xg, case["x"], atol=1e-7 * max(1.0, np.abs(case["x"]).max()))
    assert np.array_equal(np.flatnonzero(xg), np.flatnonzero(case["x"]))
    ctx.close()


def test_zero_solution_at_threshold():
    # lam1 = ||A^T b||_inf computed on the device by the same stream that forms u = A^T y
    p = synth.make_problem(60, 500, k=5, seed=4)
    ctx = pkg.Context(p.At)
    _, res, done = ctx.path(p.b, 0.6, [1.0, 1.3])
    assert done == 2 and all(r.active == 0 and r.status == pkg.OK for r in res)
    X, res, done = ctx.path(p.b, 0.6, [1.0])
    assert torch.count_nonzero(X).item() == 0
    ctx.close()


def test_orthonormal_closed_form_gpu():
    rng = np.random.default_rng(9)
    m, n = 40, 25
    Q, _ = np.linalg.qr(rng.normal(size=(m, n)))
    At = np.ascontiguousarray(Q.T)
    b = rng.normal(size=m) * 3
    l1, l2 = 0.8, 1.0
    o = pkg.ssnal_en_default_options(tol=1e-9)
    ctx = pkg.Context(At, options=o)
    x, _, res = ctx.solve(b, l1, l2)
    np.testing.assert_allclose(x.cpu().numpy(), C.soft(At @ b, l1) / (1 + l2), atol=1e-8)
    ctx.close()


def test_path_parity_small():
    p = synth.make_problem(80, 3000, k=8, seed=12, block=20, rho=0.7)
    grid = synth.path_grid(10, 0.05)
    ctx = pkg.Context(p.At)
    X, res, done = ctx.path(p.b, 0.6, grid)
    ro = R.path(p.At, p.b, 0.6, grid)
    assert done == len(grid)
    Xg = X.cpu().numpy()
    for k, rk in enumerate(ro):
        assert res[k].status == pkg.OK
        assert_parity(p.At, p.b, rk.lam1, rk.lam2, Xg[k], rk)
    ctx.close()


def test_path_max_active_truncates():
    p = synth.make_problem(80, 3000, k=8, seed=12, block=20, rho=0.7)
    grid = synth.path_grid(10, 0.05)
    o = pkg.ssnal_en_default_options(max_active=5)
    ctx = pkg.Context(p.At, options=o)
    _, res, done = ctx.path(p.b, 0.6, grid)
    ro = R.path(p.At, p.b, 0.6, grid, max_active=5)
    assert done == len(ro)
    assert res[done - 1].active >= 5 and all(r.active < 5 for r in res[:done - 1])
    ctx.close()


def test_path_host_matches_device_path():
    p = synth.make_problem(50, 1000, k=5, seed=3)
    grid = synth.path_grid(5, 0.1)
    ctx = pkg.Context(p.At)
    X, res, done = ctx.path(p.b, 0.7, grid)
    Xh = np.zeros((len(grid), p.n))
    st, resh, doneh = pkg.ssnal_en_path_host(ctx.ctx, p.b, 0.7, grid, Xh)
    assert done == doneh
    np.testing.assert_array_equal(Xh, X.cpu().numpy())  # same kernels, same order: bitwise
    ctx.close()


@pytest.mark.parametrize("precision", [0, 2, 3])
def test_config1_parity_both_streams(precision):
    p = synth.config1()
    lam1, lam2 = R.lambdas(p.At, p.b, p.alpha, p.c)
    xg, yg, res, ro = _solve_both(p, lam1, lam2, options=pkg.ssnal_en_default_options(precision=precision))
    assert res.status == pkg.OK
    assert_parity(p.At, p.b, lam1, lam2, xg, ro)
    assert res.al_iters == ro.al_iters


def test_bitwise_repeatable():
    p = synth.make_problem(100, 4000, k=10, seed=8, block=20, rho=0.5)
    lam1, lam2 = R.lambdas(p.At, p.b, 0.7, 0.3)
    ctx = pkg.Context(p.At)
    x1, y1, r1 = ctx.solve(p.b, lam1, lam2)
    x2, y2, r2 = ctx.solve(p.b, lam1, lam2)
    assert torch.equal(x1, x2) and torch.equal(y1, y2)
    assert (r1.newton_iters, r1.ls_trials) == (r2.newton_iters, r2.ls_trials)
    ctx.close()


def test_line_search_fallback_pass_matches_fused():
    # ls_fused = 1 puts every trial after the first into the vector-only pass
    p = synth.make_problem(60, 2000, k=6, seed=13)
    lam1, lam2 = R.lambdas(p.At, p.b, 0.8, 0.3)
    ctx = pkg.Context(p.At)
    x1, _, r1 = ctx.solve(p.b, lam1, lam2)
    ctx.set_options(pkg.ssnal_en_default_options(ls_fused=1))
    x2, _, r2 = ctx.solve(p.b, lam1, lam2)
    assert r1.ls_trials == r2.ls_trials and r1.newton_iters == r2.newton_iters
    np.testing.assert_allclose(x1.cpu().numpy(), x2.cpu().numpy(), rtol=0, atol=1e-12)
    ctx.close()


def test_enoconv_returns_iterate():
    p = synth.make_problem(60, 2000, k=6, seed=13)
    lam1, lam2 = R.lambdas(p.At, p.b, 0.8, 0.3)
    ctx = pkg.Context(p.At, options=pkg.ssnal_en_default_options(max_al=1))
    x, _, res = ctx.solve(p.b, lam1, lam2)
    assert res.status == pkg.ENOCONV and res.al_iters == 1
    assert np.isfinite(res.kkt1) and np.isfinite(res.kkt3)
    ctx.close()


def test_invalid_lambda_rejected():
    p = synth.make_problem(10, 50, k=2, seed=1)
    ctx = pkg.Context(p.At)
    for l1, l2 in [(-1.0, 1.0), (1.0, -0.5), (float("nan"), 1.0), (1.0, float("inf"))]:
        with pytest.raises(pkg.SsnalError) as e:
            ctx.solve(p.b, l1, l2)
        assert e.value.status == pkg.EINVAL
    ctx.close()


# ---------------------------------------------------------------- tracing (ssnal_en_profile)
def test_profile_times_one_stream_launch_in_eight_and_all_at_level_two():
    p = synth.make_problem(80, 3000, k=8, seed=12, block=20, rho=0.7)
    grid = synth.path_grid(10, 0.05)
    ctx = pkg.Context(p.At)
    ctx.path(p.b, 0.6, grid)  # warm-up
    torch.cuda.synchronize()
    for level2, every in ((False, 8), (True, 1)):
        pkg.ssnal_en_profile(ctx.ctx, True, True, phases=level2)
        X, res, done = ctx.path(p.b, 0.6, grid)
        prof = pkg.ssnal_en_profile(ctx.ctx, False, False)
        newton = sum(r.newton_iters for r in res[:done])  # one A^T d launch per Newton step
        assert done == len(grid) and newton > 8
        assert prof["stream_launches"] == (newton + every - 1) // every
        assert prof["stream_ms"] > 0.0
        per = prof["stream_bytes"] / prof["stream_launches"]
        assert per == pytest.approx(8.0 * 80 * 3000 + 3 * 8.0 * 3000 + 8.0 * 80)  # A once, x u t, d
        ph = pkg.ssnal_en_profile_phases(ctx.ctx)
        # one u = A^T y pass per fit in the FP64 form, every one timed, except the first point:
        # its initial u = A^T(-b) comes from the lambda_max pass
        assert ph["u_refresh"][1] == done - 1
        if level2:
            assert all(n > 0 for _, n in ph.values())
    ctx.close()


@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_path_first_point_equals_a_cold_solve_bitwise(storage):
    # the path's first point takes its initial u = A^T(-b) as the negation of the
    # ||A^T b||_inf pass (the pass is odd in its vector); a cold solve runs the pass itself
    p = synth.make_problem(90, 4000, k=8, seed=31, block=20, rho=0.6, dtype=np.float32)
    if storage == "bf16":
        ctx = pkg.Context(synth.to_bf16_bits(p.At), dtype=pkg.BF16,
                          options=pkg.ssnal_en_default_options(precision=1))
    else:
        ctx = pkg.Context(p.At.astype(np.float64))
    alpha, c = 0.7, 0.3
    X, res, done = ctx.path(p.b, alpha, [c])
    u = torch.empty(ctx.n, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(p.b), u)  # A^T b, the arithmetic of the lambda_max pass
    gmax = u.abs().max().item()
    lam1, lam2 = c * gmax, (1.0 - alpha) / alpha * c * gmax
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    st, r = pkg.ssnal_en_solve(ctx.ctx, dev(p.b), lam1, lam2, x)
    ctx.close()
    assert st == pkg.OK and res[0].status == pkg.OK
    assert (res[0].lambda1, res[0].lambda2) == (lam1, lam2)
    np.testing.assert_array_equal(X[0].cpu().numpy(), x.cpu().numpy())
    assert res[0].newton_iters == r.newton_iters
