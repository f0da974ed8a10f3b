"""GPU parity of the conjugate-gradient Newton solve (Algorithm 1 step (1); Sec. 3.2 proposes
CG when m and r both exceed 1e4): the device iteration against the oracle's
newton_direction_cg and the direct solve, and whole fits with the CG switch moved down
(options.cg_above) on both sides."""
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


@pytest.mark.parametrize("m,r,kappa", [(30, 1, 0.05), (30, 29, 0.05), (30, 31, 0.05), (100, 250, 0.05),
                                       (257, 65, 0.5), (500, 120, 0.05), (1000, 999, 0.01), (2048, 3000, 0.002),
                                       (4096, 700, 0.01)])
def test_cg_newton_direction_matches_the_oracle(m, r, kappa):
    rng = np.random.default_rng(m + 7 * r)
    At = rng.normal(size=(r + 10, m))
    J = np.arange(r, dtype=np.int32)
    g = rng.normal(size=m)
    ctx = pkg.Context(At, options=pkg.ssnal_en_default_options(cg_above=0))
    gd = torch.empty(m, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_grad(ctx.ctx, dev(J, torch.int32), dev(np.zeros(r)), r, dev(-g), dev(np.zeros(m)), gd)
    d = torch.empty(m, dtype=torch.float64, device="cuda")
    st = pkg.ssnal_en_op_newton(ctx.ctx, r, kappa, dev(g), d)
    ctx.close()
    assert st == pkg.OK
    dg = d.cpu().numpy()
    dcg, it = R.newton_direction_cg(At[J], g, kappa, rtol=1e-10)
    ref = R.newton_direction(At[J], g, kappa)
    # both stop at ||V d + g|| <= 1e-10 ||g||; V's condition number here is below ~1e3
    scale = np.abs(ref).max()
    assert np.abs(dg - ref).max() <= 1e-7 * scale
    assert np.abs(dg - dcg).max() <= 1e-7 * scale
    V = np.eye(m) + kappa * At[J].T @ At[J]
    assert np.linalg.norm(V @ dg + g) <= 2e-10 * np.linalg.norm(g)


@pytest.mark.parametrize("m,n,alpha,c,seed,cg_above", [(40, 160, 0.7, 0.3, 21, 0), (60, 300, 0.6, 0.2, 40, 50),
                                                      (120, 2000, 0.8, 0.1, 3, 0)])
def test_fit_with_cg_matches_the_oracle(m, n, alpha, c, seed, cg_above):
    # cg_above = 0: every Newton step by CG; 50: steps with r > 50 by CG, the rest direct
    p = synth.make_problem(m, n, k=max(4, m // 10), seed=seed, block=10, rho=0.5)
    lam1, lam2 = R.lambdas(p.At, p.b, alpha, c)
    ctx = pkg.Context(p.At, options=pkg.ssnal_en_default_options(cg_above=cg_above))
    x, _, res = ctx.solve(p.b, lam1, lam2)
    ctx.close()
    ro = R.solve(p.At, p.b, lam1, lam2, opts=R.Options(cg_above=cg_above))
    assert ro.converged and res.status == pkg.OK
    assert res.cg_iters > 0
    assert_parity(p.At, p.b, lam1, lam2, x.cpu().numpy(), ro)
