"""GPU parity at the benchmarked sizes (marked slow: the oracle runs for minutes here).

  * the FP64 regularization path of the path configuration (m = 500, n = 1e5, 20 points)
    against oracle.path, point by point;
  * the precision configuration (m = 1000, n = 1e6) at alpha 0.5 and 0.9: the mixed form
    (BF16 storage) against the oracle on the stored BF16 values (solver error, at the FP64
    bars) and against the oracle on the FP32 matrix (BF16 storage error, stated), and the
    FP64 form against the oracle on the FP32 matrix;
  * a genotype fit at m = 2000 (int8 codes), and a fit whose panel exceeds the size the
    cluster GEMV serves (m * panel capacity > 2^22: the beyond-L2 panel GEMV).
Bars as in test_gpu_parity."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import paper_2006_03970_gb300 as pkg  # noqa: E402
from oracle import checkers as C  # noqa: E402
from oracle import ssnal_en_ref as R  # noqa: E402
from paper_2006_03970_gb300 import synth  # noqa: E402

from test_gpu_parity import assert_parity  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_03970_gb300 import build
    build.build()
    pkg.load_library()


def test_path_configuration_full_path_matches_the_oracle():
    p = synth.config2()
    grid = synth.path_grid(20, 0.05)
    ctx = pkg.Context(p.At)
    X, res, done = ctx.path(p.b, 0.6, grid)
    ctx.close()
    ro = R.path(p.At, p.b, 0.6, grid)
    assert done == len(grid) == len(ro)
    Xg = X.cpu().numpy()
    for k, rk in enumerate(ro):
        assert res[k].status == pkg.OK and rk.converged
        assert res[k].kkt1 <= 1e-6 and res[k].kkt3 <= 1e-6
        assert_parity(p.At, p.b, rk.lam1, rk.lam2, Xg[k], rk)
    assert np.count_nonzero(Xg[0]) == 0  # c = 1: the null model


@pytest.fixture(scope="module")
def precision_workload():
    p = synth.config3()
    bits = synth.to_bf16_bits(p.At)
    return p, bits


@pytest.mark.parametrize("alpha", [0.5, 0.9])
def test_precision_configuration_both_forms_match_the_oracle(precision_workload, alpha):
    p, bits = precision_workload
    c = 0.3
    b = torch.as_tensor(p.b, device="cuda")
    ctx = pkg.Context(bits, dtype=pkg.BF16, options=pkg.ssnal_en_default_options(precision=1))
    Xm, res_m, _ = ctx.path(p.b, alpha, [c])
    ctx.close()
    xm = Xm[0].cpu().numpy()
    del Xm
    assert res_m[0].status == pkg.OK and res_m[0].kkt1 <= 1e-6 and res_m[0].kkt3 <= 1e-6
    # (i) solver error: the oracle on the stored values
    Ab = np.ascontiguousarray(synth.bf16_bits_to_f32(bits), dtype=np.float64)
    l1, l2 = R.lambdas(Ab, p.b, alpha, c)
    ro = R.solve(Ab, p.b, l1, l2)
    assert ro.converged
    assert_parity(Ab, p.b, l1, l2, xm, ro)
    del Ab
    # (ii) the FP64 form against the oracle on the FP32 matrix, and the BF16 storage error
    Af = np.ascontiguousarray(p.At, dtype=np.float64)
    ctx = pkg.Context(Af)
    Xf, res_f, _ = ctx.path(b, alpha, [c])
    ctx.close()
    xf = Xf[0].cpu().numpy()
    del Xf
    assert res_f[0].status == pkg.OK
    l1, l2 = R.lambdas(Af, p.b, alpha, c)
    rf = R.solve(Af, p.b, l1, l2)
    assert rf.converged
    assert_parity(Af, p.b, l1, l2, xf, rf)
    storage = np.abs(xm - rf.x).max() / np.abs(rf.x).max()
    P_m = C.primal_objective(Af, p.b, xm, l1, l2)
    P_or = C.primal_objective(Af, p.b, rf.x, l1, l2)
    # BF16 keeps 8 significant bits of each entry: the solutions differ by about 1e-3
    # relative, the objective by about 1e-6 relative
    assert storage <= 1e-2, storage
    assert abs(P_m - P_or) <= 1e-5 * abs(P_or)


def test_genotype_fit_at_m_2000_matches_the_oracle():
    codes, mean, scale = synth.genotype_matrix(2000, 6000, seed=61)
    As = (codes.astype(np.float64) - mean.astype(np.float64)[:, None]) * scale.astype(np.float64)[:, None]
    rng = np.random.default_rng(62)
    x = np.zeros(6000)
    idx = rng.choice(6000, size=30, replace=False)
    x[idx] = rng.choice([-1.0, 1.0], size=30) * rng.uniform(0.5, 2.0, size=30)
    Ax = As.T @ x
    b = Ax + np.sqrt(Ax.var() / 2.0) * rng.normal(size=2000)
    lam1, lam2 = R.lambdas(As, b, 0.8, 0.3)
    A, _ = pkg.device_matrix(codes, pkg.I8_GENO)
    cm = torch.as_tensor(mean, device="cuda")
    cs = torch.as_tensor(scale, device="cuda")
    ctx = pkg.Context(A, m=2000, dtype=pkg.I8_GENO, col_mean=cm, col_scale=cs)
    xg, _, res = ctx.solve(b, lam1, lam2)
    ctx.close()
    ro = R.solve(As, b, lam1, lam2)
    assert res.status == pkg.OK and ro.converged
    assert_parity(As, b, lam1, lam2, xg.cpu().numpy(), ro)


def test_fit_through_the_beyond_l2_panel_gemv():
    # m = 2100: the panel capacity starts at m, m * capacity > 2^22, so every A_J w and
    # A_J q of this fit runs in the beyond-L2 GEMV (row tiles x column chunks)
    p = synth.make_problem(2100, 3000, k=40, seed=71, block=20, rho=0.5)
    lam1, lam2 = R.lambdas(p.At, p.b, 0.7, 0.2)
    ctx = pkg.Context(p.At)
    x, _, res = ctx.solve(p.b, lam1, lam2)
    ctx.close()
    ro = R.solve(p.At, p.b, lam1, lam2)
    assert res.status == pkg.OK and ro.converged
    assert max(ro.r_history) > 0
    assert_parity(p.At, p.b, lam1, lam2, x.cpu().numpy(), ro)
