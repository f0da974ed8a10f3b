"""GPU parity of BF16 / FP32 storage of A (the precision form of the method).

The oracle solves the same problem on the *stored* values upcast to FP64, so any
difference is solver error, not storage error:
  * every pass with float-float accumulation (precision 0) meets the FP64-path bars;
  * the mixed mode (precision 1: FP32-accumulated Newton passes, u = A^T y recomputed in
    float-float before each SsN stopping test) still converges to KKT <= 1e-6 in FP64,
    and its x is compared with the oracle's at a tolerance derived from that residual.
Kernel-level tests bound the stream error from the arithmetic.
"""
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


def stored(At32, dtype):
    """(device-storage array, the stored values as FP64)."""
    if dtype == pkg.BF16:
        bits = synth.to_bf16_bits(At32)
        return bits, synth.bf16_bits_to_f32(bits).astype(np.float64)
    a = np.ascontiguousarray(At32, dtype=np.float32)
    return a, a.astype(np.float64)


# ---------------------------------------------------------------- a1 on BF16 / FP32
@pytest.mark.parametrize("dtype", [pkg.BF16, pkg.F32])
@pytest.mark.parametrize("m,n", [(1, 1), (7, 33), (63, 64), (64, 65), (100, 2000), (513, 4097), (2000, 777)])
def test_stream_low_precision_storage(dtype, m, n):
    rng = np.random.default_rng(m * 11 + n)
    At32 = rng.normal(size=(n, m)).astype(np.float32)
    data, At = stored(At32, dtype)
    y = rng.normal(size=m)
    ref = At @ y
    mag = np.abs(At) @ np.abs(y)
    ctx = pkg.Context(data, dtype=dtype)
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    # u = A^T y: float-float, products of the stored values exact (same bound as the FP64 stream)
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(y), u)
    bound = (2.0 ** -45 + m * 2.0 ** -47) * mag + 1e-300
    assert np.all(np.abs(u.cpu().numpy() - ref) <= bound)
    # mixed mode Newton pass: y split to FP32 (2^-24) and m FP32 roundings of the running sums
    ctx.set_options(pkg.ssnal_en_default_options(precision=1))
    t = torch.empty(n, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_at_d(ctx.ctx, dev(y), t)
    bound32 = (m + 2) * 2.0 ** -24 * mag + 1e-300
    err = np.abs(t.cpu().numpy() - ref)
    assert np.all(err <= bound32)
    # and u = A^T y stays float-float in that mode
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(y), u)
    assert np.all(np.abs(u.cpu().numpy() - ref) <= bound)
    ctx.close()


def test_stream_bf16_padding_rows_ignored():
    rng = np.random.default_rng(9)
    m, n = 13, 200  # lda = 16: three padding rows
    At32 = rng.normal(size=(n, m)).astype(np.float32)
    data, At = stored(At32, pkg.BF16)
    A, _ = pkg.device_matrix(data, pkg.BF16)
    A[:, m:] = 0x7FC0  # BF16 NaN in the padding rows
    ctx = pkg.Context(A, m=m, dtype=pkg.BF16)
    y = rng.normal(size=m)
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(y), u)
    assert torch.isfinite(u).all()
    assert np.allclose(u.cpu().numpy(), At @ y, rtol=1e-12, atol=1e-12)
    ctx.close()


# ---------------------------------------------------------------- whole fits
def _problem(m, n, seed, block, rho, k, snr):
    p = synth.make_problem(m, n, k=k, seed=seed, block=block, rho=rho, snr=snr, alpha=0.5)
    return p


@pytest.mark.parametrize("dtype", [pkg.BF16, pkg.F32])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,n,alpha,c,seed,block,rho", [
    (120, 6000, 0.5, 0.3, 31, 50, 0.5), (120, 6000, 0.9, 0.3, 32, 50, 0.5), (60, 900, 0.7, 0.1, 33, 1, 0.0),
    (300, 2500, 0.9, 0.3, 34, 50, 0.5)])
def test_fit_low_precision_storage(dtype, precision, m, n, alpha, c, seed, block, rho):
    p = synth.make_problem(m, n, k=max(5, m // 20), seed=seed, block=block, rho=rho, snr=3.0, alpha=alpha)
    data, At = stored(p.At.astype(np.float32), dtype)
    lam1, lam2 = R.lambdas(At, p.b, alpha, c)
    ctx = pkg.Context(data, dtype=dtype, options=pkg.ssnal_en_default_options(precision=precision))
    x, y, res = ctx.solve(p.b, lam1, lam2)
    xg = x.cpu().numpy()
    ctx.close()
    ro = R.solve(At, p.b, lam1, lam2)
    assert res.status == pkg.OK and ro.converged
    assert res.kkt1 <= 1e-6 and res.kkt3 <= 1e-6
    # the residuals the solver reported agree with an independent FP64 evaluation on the stored values
    kkt = C.kkt_violation(At, p.b, xg, lam1, lam2)
    assert kkt <= 1e-5 * max(1.0, np.abs(At @ p.b).max())
    P_or = C.primal_objective(At, p.b, ro.x, lam1, lam2)
    P_gpu = C.primal_objective(At, p.b, xg, lam1, lam2)
    xmax = np.abs(ro.x).max()
    if precision == 0:
        assert abs(P_gpu - P_or) <= 1e-9 * max(1.0, abs(P_or))
        assert np.abs(xg - ro.x).max() <= 1e-6 * xmax
    else:
        # both iterates meet KKT <= 1e-6; by strong convexity (modulus lam2) the objective gap and
        # the distance between them are of the order of the residuals
        assert abs(P_gpu - P_or) <= 1e-6 * max(1.0, abs(P_or))
        assert np.abs(xg - ro.x).max() <= 1e-3 * xmax
    big = np.abs(ro.x) > 1e-4 * xmax
    assert np.all(xg[big] != 0.0)


def test_bf16_path_matches_oracle_path():
    p = synth.make_problem(100, 3000, k=5, seed=41, block=50, rho=0.5, snr=3.0, alpha=0.6)
    data, At = stored(p.At.astype(np.float32), pkg.BF16)
    grid = synth.path_grid(6, 0.1)
    ctx = pkg.Context(data, dtype=pkg.BF16, options=pkg.ssnal_en_default_options(precision=1))
    X, res, done = ctx.path(p.b, 0.6, grid)
    ctx.close()
    assert done == len(grid)
    ro = R.path(At, p.b, 0.6, grid)
    Xg = X.cpu().numpy()
    for k, rk in enumerate(ro):
        assert res[k].status == pkg.OK
        assert res[k].kkt1 <= 1e-6 and res[k].kkt3 <= 1e-6
        xmax = np.abs(rk.x).max()
        if xmax == 0:
            assert np.all(Xg[k] == 0.0)
        else:
            assert np.abs(Xg[k] - rk.x).max() <= 1e-3 * xmax


# ---------------------------------------------------------------- int8 genotype codes
def genotype_problem(m, n, seed, k=6, snr=2.0):
    codes, mean, scale = synth.genotype_matrix(m, n, seed=seed)
    As = (codes.astype(np.float64) - mean.astype(np.float64)[:, None]) * scale.astype(np.float64)[:, None]
    rng = np.random.default_rng(seed + 1)
    k = min(k, n)
    x = np.zeros(n)
    idx = rng.choice(n, size=k, replace=False)
    x[idx] = rng.choice([-1.0, 1.0], size=k) * rng.uniform(0.5, 2.0, size=k)
    Ax = As.T @ x
    b = Ax + np.sqrt(Ax.var() / snr) * rng.normal(size=m)
    return codes, mean, scale, As, b


def genotype_context(codes, mean, scale, precision):
    m = codes.shape[1]
    A, _ = pkg.device_matrix(codes, pkg.I8_GENO)
    cm, cs = dev(mean, torch.float32), dev(scale, torch.float32)
    return pkg.Context(A, m=m, dtype=pkg.I8_GENO, options=pkg.ssnal_en_default_options(precision=precision),
                       col_mean=cm, col_scale=cs)


@pytest.mark.parametrize("m,n", [(1, 1), (5, 40), (127, 129), (128, 300), (300, 5000), (2000, 511)])
def test_stream_genotype_codes(m, n):
    codes, mean, scale, As, _ = genotype_problem(m, n, seed=m + n)
    rng = np.random.default_rng(m)
    y = rng.normal(size=m)
    ref = As @ y
    s = np.abs(scale.astype(np.float64))
    mag = s * (np.abs(codes.astype(np.float64)) @ np.abs(y) + np.abs(mean.astype(np.float64)) * np.abs(y).sum())
    ctx = genotype_context(codes, mean, scale, 0)
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_at_y(ctx.ctx, dev(y), u)
    # float-float code * y sums, then scale * (sum - mean * sum(y)) in FP64
    bound = (2.0 ** -44 + m * 2.0 ** -46) * mag + 1e-300
    assert np.all(np.abs(u.cpu().numpy() - ref) <= bound)
    ctx.set_options(pkg.ssnal_en_default_options(precision=1))
    t = torch.empty(n, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_at_d(ctx.ctx, dev(y), t)
    assert np.all(np.abs(t.cpu().numpy() - ref) <= (m + 4) * 2.0 ** -24 * mag + 1e-300)
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,n,alpha,c,seed", [(150, 4000, 0.7, 0.3, 51), (400, 3000, 0.95, 0.2, 52)])
def test_fit_genotype_codes(precision, m, n, alpha, c, seed):
    codes, mean, scale, As, b = genotype_problem(m, n, seed)
    lam1, lam2 = R.lambdas(As, b, alpha, c)
    ctx = genotype_context(codes, mean, scale, precision)
    x, y, res = ctx.solve(b, lam1, lam2)
    xg = x.cpu().numpy()
    ctx.close()
    ro = R.solve(As, b, lam1, lam2)
    assert res.status == pkg.OK and ro.converged
    assert res.kkt1 <= 1e-6 and res.kkt3 <= 1e-6
    xmax = np.abs(ro.x).max()
    P_or = C.primal_objective(As, b, ro.x, lam1, lam2)
    P_gpu = C.primal_objective(As, b, xg, lam1, lam2)
    if precision == 0:
        assert abs(P_gpu - P_or) <= 1e-9 * max(1.0, abs(P_or))
        assert np.abs(xg - ro.x).max() <= 1e-6 * xmax
    else:
        assert abs(P_gpu - P_or) <= 1e-6 * max(1.0, abs(P_or))
        assert np.abs(xg - ro.x).max() <= 1e-3 * xmax


# ---------------------------------------------------------------- 2-bit genotype codes (four per byte)
def genotype_context_2bit(codes, mean, scale, precision):
    m = codes.shape[1]
    A, _ = pkg.device_matrix(codes, pkg.I2_GENO)
    cm, cs = dev(mean, torch.float32), dev(scale, torch.float32)
    return pkg.Context(A, m=m, dtype=pkg.I2_GENO, options=pkg.ssnal_en_default_options(precision=precision),
                       col_mean=cm, col_scale=cs)


@pytest.mark.parametrize("m,n", [(1, 1), (5, 40), (127, 129), (512, 300), (513, 300), (1000, 5000), (2000, 511)])
def test_stream_genotype_codes_2bit(m, n):
    codes, mean, scale, As, _ = genotype_problem(m, n, seed=m + n)
    rng = np.random.default_rng(m)
    y = rng.normal(size=m)
    ref = As @ y
    s = np.abs(scale.astype(np.float64))
    mag = s * (np.abs(codes.astype(np.float64)) @ np.abs(y) + np.abs(mean.astype(np.float64)) * np.abs(y).sum())
    ctx2 = genotype_context_2bit(codes, mean, scale, 0)
    ctx8 = genotype_context(codes, mean, scale, 0)
    u2 = torch.empty(n, dtype=torch.float64, device="cuda")
    u8 = torch.empty(n, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_at_y(ctx2.ctx, dev(y), u2)
    pkg.ssnal_en_op_at_y(ctx8.ctx, dev(y), u8)
    bound = (2.0 ** -44 + m * 2.0 ** -46) * mag + 1e-300
    u2h = u2.cpu().numpy()
    assert np.all(np.abs(u2h - ref) <= bound)
    # the int8 and 2-bit passes sum the same exact products in a different order (512 rows
    # per box against 128): both float-float, they agree to the same bound
    assert np.all(np.abs(u2h - u8.cpu().numpy()) <= 2 * bound)
    for c in (ctx2, ctx8):
        c.set_options(pkg.ssnal_en_default_options(precision=1))
    t2 = torch.empty(n, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_at_d(ctx2.ctx, dev(y), t2)
    assert np.all(np.abs(t2.cpu().numpy() - ref) <= (m + 4) * 2.0 ** -24 * mag + 1e-300)
    ctx2.close()
    ctx8.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,n,alpha,c,seed", [(150, 4000, 0.7, 0.3, 51), (400, 3000, 0.95, 0.2, 52),
                                              (2000, 3000, 0.8, 0.3, 53)])
def test_fit_genotype_codes_2bit(precision, m, n, alpha, c, seed):
    codes, mean, scale, As, b = genotype_problem(m, n, seed)
    lam1, lam2 = R.lambdas(As, b, alpha, c)
    ctx = genotype_context_2bit(codes, mean, scale, precision)
    x, y, res = ctx.solve(b, lam1, lam2)
    xg = x.cpu().numpy()
    ctx.close()
    ro = R.solve(As, b, lam1, lam2)
    assert res.status == pkg.OK and ro.converged
    assert res.kkt1 <= 1e-6 and res.kkt3 <= 1e-6
    xmax = np.abs(ro.x).max()
    P_or = C.primal_objective(As, b, ro.x, lam1, lam2)
    P_gpu = C.primal_objective(As, b, xg, lam1, lam2)
    if precision == 0:
        assert abs(P_gpu - P_or) <= 1e-9 * max(1.0, abs(P_or))
        assert np.abs(xg - ro.x).max() <= 1e-6 * xmax
    else:
        assert abs(P_gpu - P_or) <= 1e-6 * max(1.0, abs(P_or))
        assert np.abs(xg - ro.x).max() <= 1e-3 * xmax
