"""Serving loop: requests on resident matrices, admitted while others run.

Every request must give bitwise the result of ssnal_en_solve on its own (same kernels,
same order within the request), whatever else is in flight; the results also meet the
KKT tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2006_03970_gb300 as pkg  # noqa: E402
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


def resident_matrices():
    """(device matrix tuple, stored values as FP64 (n, m))."""
    out = []
    p = synth.make_problem(120, 3000, k=5, seed=61, block=50, rho=0.5, dtype=np.float32)
    A, m = pkg.device_matrix(p.At.astype(np.float32), pkg.F32)
    out.append(((A, m, pkg.F32, None, None), p.At.astype(np.float32).astype(np.float64)))
    codes, mean, scale = synth.genotype_matrix(200, 4000, seed=62)
    A, m = pkg.device_matrix(codes, pkg.I8_GENO)
    vals = (codes.astype(np.float64) - mean.astype(np.float64)[:, None]) * scale.astype(np.float64)[:, None]
    out.append(((A, m, pkg.I8_GENO, dev(mean, torch.float32), dev(scale, torch.float32)), vals))
    q = synth.make_problem(80, 2000, k=5, seed=63, dtype=np.float32)
    bits = synth.to_bf16_bits(q.At.astype(np.float32))
    A, m = pkg.device_matrix(bits, pkg.BF16)
    out.append(((A, m, pkg.BF16, None, None), synth.bf16_bits_to_f32(bits).astype(np.float64)))
    return out


def requests(mats, count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(count):
        k = int(rng.integers(0, len(mats)))
        vals = mats[k][1]
        n, m = vals.shape
        x = np.zeros(n)
        idx = rng.choice(n, size=8, replace=False)
        x[idx] = rng.choice([-1.0, 1.0], size=8) * rng.uniform(0.5, 2.0, size=8)
        ax = vals.T @ x
        b = ax + np.sqrt(ax.var() / 2.0) * rng.normal(size=m)
        alpha, c = rng.uniform(0.5, 0.999), rng.uniform(0.1, 0.8)
        lmax = np.abs(vals @ b).max()
        reqs.append((k, b, c * lmax, (1 - alpha) / alpha * c * lmax))
    return reqs


@pytest.mark.parametrize("precision", [0, 1])
def test_requests_in_the_mix_match_alone(precision):
    mats = resident_matrices()
    opts = pkg.ssnal_en_default_options(precision=precision)
    reqs = requests(mats, 30, 7 + precision)
    srv = pkg.Server([d for d, _ in mats], workers=4, options=opts)
    tickets = [srv.submit(k, b, l1, l2) for k, b, l1, l2 in reqs]
    got = [srv.poll(t, k, wait=True) for t, (k, _, _, _) in zip(tickets, reqs)]
    srv.close()
    # each request alone, on a fresh context of its matrix
    ctxs = []
    for (A, m, dtype, cm, cs), _ in mats:
        ctxs.append(pkg.Context(A, m=m, dtype=dtype, options=opts, col_mean=cm, col_scale=cs))
    for (k, b, l1, l2), (x, res, times) in zip(reqs, got):
        assert res.status == pkg.OK and res.kkt1 <= 1e-6 and res.kkt3 <= 1e-6
        assert times[0] <= times[1] <= times[2]
        xa = torch.zeros(ctxs[k].n, dtype=torch.float64, device="cuda")
        st, ra = pkg.ssnal_en_solve(ctxs[k].ctx, dev(b), l1, l2, xa)
        assert st == pkg.OK
        np.testing.assert_array_equal(x, xa.cpu().numpy())
        assert ra.newton_iters == res.newton_iters
    for c in ctxs:
        c.close()


def test_admission_bound_still_serves_everything():
    mats = resident_matrices()
    reqs = requests(mats, 10, 3)
    srv = pkg.Server([d for d, _ in mats], workers=4, max_bytes=1)  # at most one request in flight
    tickets = [srv.submit(k, b, l1, l2) for k, b, l1, l2 in reqs]
    got = [srv.poll(t, k, wait=True) for t, (k, _, _, _) in zip(tickets, reqs)]
    srv.close()
    spans = sorted((times[1], times[2]) for _, _, times in got)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-9  # one at a time: no two solves overlap
    assert all(res.status == pkg.OK for _, res, _ in got)


@pytest.mark.parametrize("group", [1, 8])
def test_merged_groups_match_alone(group):
    # many requests on the same matrices, queued at once: with group 8 the workers advance
    # up to eight fits of one matrix together and merge their passes over A
    mats = resident_matrices()
    opts = pkg.ssnal_en_default_options(precision=1)
    reqs = requests(mats, 40, 11)
    srv = pkg.Server([d for d, _ in mats], workers=2, options=opts, group=group)
    tickets = [srv.submit(k, b, l1, l2) for k, b, l1, l2 in reqs]
    got = [srv.poll(t, k, wait=True) for t, (k, _, _, _) in zip(tickets, reqs)]
    srv.close()
    ctxs = [pkg.Context(A, m=m, dtype=dtype, options=opts, col_mean=cm, col_scale=cs)
            for (A, m, dtype, cm, cs), _ in mats]
    for (k, b, l1, l2), (x, res, times) in zip(reqs, got):
        assert res.status == pkg.OK and res.kkt1 <= 1e-6 and res.kkt3 <= 1e-6
        xa = torch.zeros(ctxs[k].n, dtype=torch.float64, device="cuda")
        st, ra = pkg.ssnal_en_solve(ctxs[k].ctx, dev(b), l1, l2, xa)
        np.testing.assert_array_equal(x, xa.cpu().numpy())
    for c in ctxs:
        c.close()
