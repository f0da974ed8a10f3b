"""Fits that share one matrix, advanced together with their passes over A merged
(A^T [d_1 ... d_k], one pass for up to four fits, each with its own fused line search):
every fit must give bitwise the result of ssnal_en_solve on its own, with fewer passes
over A than Newton steps, for every storage type whose Newton passes accumulate in FP32;
and the results meet the oracle's bars for the mixed form."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2006_03970_gb300 as pkg  # noqa: E402
from oracle import checkers as C  # noqa: E402
from oracle import ssnal_en_ref as R  # noqa: E402
from paper_2006_03970_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_03970_gb300 import build
    build.build()
    pkg.load_library()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def stored_matrix(kind, m, n, seed):
    """(device tensor, m, dtype, col_mean, col_scale, stored values as FP64 (n, m))."""
    if kind in ("i8", "i2"):
        codes, mean, scale = synth.genotype_matrix(m, n, seed=seed)
        vals = (codes.astype(np.float64) - mean.astype(np.float64)[:, None]) * scale.astype(np.float64)[:, None]
        dt = pkg.I8_GENO if kind == "i8" else pkg.I2_GENO
        A, mm = pkg.device_matrix(codes, dt)
        return A, mm, dt, dev(mean, torch.float32), dev(scale, torch.float32), vals
    p = synth.make_problem(m, n, k=5, seed=seed, block=20, rho=0.5, dtype=np.float32)
    if kind == "bf16":
        bits = synth.to_bf16_bits(p.At)
        A, mm = pkg.device_matrix(bits, pkg.BF16)
        return A, mm, pkg.BF16, None, None, synth.bf16_bits_to_f32(bits).astype(np.float64)
    if kind == "f32":
        A, mm = pkg.device_matrix(p.At, pkg.F32)
        return A, mm, pkg.F32, None, None, p.At.astype(np.float64)
    At = p.At.astype(np.float64)
    A, mm = pkg.device_matrix(At, pkg.F64)
    return A, mm, pkg.F64, None, None, At


def right_hand_sides(vals, k, seed):
    rng = np.random.default_rng(seed)
    n, m = vals.shape
    out = []
    for i in range(k):
        x = np.zeros(n)
        idx = rng.choice(n, size=8, replace=False)
        x[idx] = rng.choice([-1.0, 1.0], size=8) * rng.uniform(0.5, 2.0, size=8)
        ax = vals.T @ x
        b = ax + np.sqrt(ax.var() / 2.0) * rng.normal(size=m)
        alpha, c = rng.uniform(0.5, 0.95), rng.uniform(0.15, 0.6)
        lmax = np.abs(vals @ b).max()
        out.append((b, c * lmax, (1 - alpha) / alpha * c * lmax))
    return out


@pytest.mark.parametrize("kind,precision,k", [("bf16", 1, 4), ("bf16", 1, 7), ("f32", 1, 3), ("i8", 1, 5),
                                              ("i2", 1, 6), ("i2", 1, 1), ("f64", 0, 3)])
def test_shared_fits_match_each_fit_alone(kind, precision, k):
    m, n = (200, 5000) if kind != "i2" else (300, 6000)
    A, mm, dt, cm, cs, vals = stored_matrix(kind, m, n, seed=90 + k)
    rhs = right_hand_sides(vals, k, seed=k)
    opts = pkg.ssnal_en_default_options(precision=precision)
    ctxs = [pkg.Context(A, m=mm, dtype=dt, options=opts, col_mean=cm, col_scale=cs) for _ in range(k)]
    xs = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(k)]
    bs = [dev(b) for b, _, _ in rhs]
    inst = [(c.ctx, b, l1, l2, x, None) for c, b, (_, l1, l2), x in zip(ctxs, bs, rhs, xs)]
    st, res, passes = pkg.ssnal_en_solve_shared(inst)
    assert st == pkg.OK
    newton = sum(r.newton_iters for r in res)
    if precision == 1 and k > 1:
        assert passes < newton  # passes over A were merged
    else:
        assert passes == newton
    solo = pkg.Context(A, m=mm, dtype=dt, options=opts, col_mean=cm, col_scale=cs)
    for (b, l1, l2), x, r in zip(rhs, xs, res):
        xa = torch.zeros(n, dtype=torch.float64, device="cuda")
        sa, ra = pkg.ssnal_en_solve(solo.ctx, dev(b), l1, l2, xa)
        assert sa == pkg.OK and r.status == pkg.OK
        np.testing.assert_array_equal(x.cpu().numpy(), xa.cpu().numpy())
        assert (r.newton_iters, r.al_iters, r.ls_trials) == (ra.newton_iters, ra.al_iters, ra.ls_trials)
        assert r.kkt1 == ra.kkt1 and r.kkt3 == ra.kkt3
    solo.close()
    for c in ctxs:
        c.close()


def test_shared_fits_match_the_oracle():
    A, mm, dt, cm, cs, vals = stored_matrix("bf16", 150, 4000, seed=95)
    rhs = right_hand_sides(vals, 4, seed=5)
    opts = pkg.ssnal_en_default_options(precision=1)
    ctxs = [pkg.Context(A, m=mm, dtype=dt, options=opts) for _ in range(4)]
    xs = [torch.zeros(4000, dtype=torch.float64, device="cuda") for _ in range(4)]
    inst = [(c.ctx, dev(b), l1, l2, x, None) for c, (b, l1, l2), x in zip(ctxs, rhs, xs)]
    st, res, passes = pkg.ssnal_en_solve_shared(inst)
    assert st == pkg.OK
    for (b, l1, l2), x in zip(rhs, xs):
        ro = R.solve(vals, b, l1, l2)
        xg = x.cpu().numpy()
        P_or = C.primal_objective(vals, b, ro.x, l1, l2)
        P_g = C.primal_objective(vals, b, xg, l1, l2)
        # the mixed form's bars (FP32-accumulated Newton passes, FP64 KKT <= 1e-6)
        assert abs(P_g - P_or) <= 1e-6 * max(1.0, abs(P_or))
        assert np.abs(xg - ro.x).max() <= 1e-3 * np.abs(ro.x).max()
    for c in ctxs:
        c.close()


def test_shared_rejects_a_context_used_twice():
    A, mm, dt, cm, cs, vals = stored_matrix("bf16", 40, 300, seed=96)
    ctx = pkg.Context(A, m=mm, dtype=dt)
    x = torch.zeros(300, dtype=torch.float64, device="cuda")
    b = dev(np.ones(40))
    with pytest.raises(pkg.SsnalError):
        pkg.ssnal_en_solve_shared([(ctx.ctx, b, 1.0, 1.0, x, None), (ctx.ctx, b, 1.0, 1.0, x, None)])
    ctx.close()
