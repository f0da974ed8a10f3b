"""Batched fits of independent, uneven instances (ssnal_en_solve_batch).

Each instance of a batch is solved by the same kernels as ssnal_en_solve on its own, in a
fixed order within the instance, so its result must be bitwise the same alone and in the
batch, whatever the number of worker threads; one instance is also checked against the
oracle on its stored values.
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


def make_instances(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        m = int(np.exp(rng.uniform(np.log(30), np.log(200))))
        n = int(np.exp(rng.uniform(np.log(300), np.log(3000))))
        p = synth.make_problem(m, n, k=max(5, m // 20), seed=seed * 1000 + k, alpha=0.7, dtype=np.float32)
        At = p.At.astype(np.float32)
        lam1, lam2 = R.lambdas(At.astype(np.float64), p.b, 0.7, float(rng.uniform(0.2, 0.8)))
        out.append((At, p.b, lam1, lam2))
    return out


def test_batch_matches_single_solves_bitwise():
    probs = make_instances(24, 7)
    ctxs = [pkg.Context(At, dtype=pkg.F32) for At, _, _, _ in probs]
    bs = [dev(b) for _, b, _, _ in probs]
    # alone, one after the other
    alone = []
    for ctx, b, (At, _, l1, l2) in zip(ctxs, bs, probs):
        x = torch.zeros(At.shape[0], dtype=torch.float64, device="cuda")
        st, res = pkg.ssnal_en_solve(ctx.ctx, b, l1, l2, x)
        assert st == pkg.OK
        alone.append(x.cpu().numpy())
    for workers in (0, 3):
        xs = [torch.zeros(At.shape[0], dtype=torch.float64, device="cuda") for At, _, _, _ in probs]
        inst = [(ctx.ctx, b, l1, l2, x, None) for ctx, b, (_, _, l1, l2), x in zip(ctxs, bs, probs, xs)]
        st, res, used = pkg.ssnal_en_solve_batch(inst, workers)
        assert st == pkg.OK
        assert used in ((4, 8, 16, 32) if workers == 0 else (3,))
        for k in range(len(probs)):
            assert res[k].status == pkg.OK and res[k].kkt1 <= 1e-6 and res[k].kkt3 <= 1e-6
            np.testing.assert_array_equal(xs[k].cpu().numpy(), alone[k])
    # one instance against the oracle on the stored FP32 values
    At, b, l1, l2 = probs[5]
    ro = R.solve(At.astype(np.float64), b, l1, l2)
    P_or = C.primal_objective(At.astype(np.float64), b, ro.x, l1, l2)
    P_gpu = C.primal_objective(At.astype(np.float64), b, alone[5], l1, l2)
    assert abs(P_gpu - P_or) <= 1e-9 * max(1.0, abs(P_or))
    assert np.abs(alone[5] - ro.x).max() <= 1e-6 * np.abs(ro.x).max()
    for ctx in ctxs:
        ctx.close()


def test_batch_rejects_shared_context():
    At, b, l1, l2 = make_instances(1, 3)[0]
    ctx = pkg.Context(At, dtype=pkg.F32)
    bd = dev(b)
    x1 = torch.zeros(At.shape[0], dtype=torch.float64, device="cuda")
    x2 = torch.zeros_like(x1)
    with pytest.raises(pkg.SsnalError):
        pkg.ssnal_en_solve_batch([(ctx.ctx, bd, l1, l2, x1, None), (ctx.ctx, bd, l1, l2, x2, None)], 2)
    ctx.close()
