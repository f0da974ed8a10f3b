"""The device-resident batched solver (ssnal_en_solve_batch_resident): one persistent kernel,
each CTA running whole fits (Algorithm 1) from a device work queue.  Every fit must meet the
FP64 oracle's bars on its FP32-stored matrix; the tuned loads in flight must not change any
result; fits the kernel hands back (FP32 Newton solve failed or not contracting) must still
match the oracle through the regular path."""
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


def make_fits(count, m_range, n_range, seed, warm=False):
    rng = np.random.default_rng(seed)
    probs, fits = [], []
    for i in range(count):
        m = int(rng.integers(*m_range))
        n = int(rng.integers(*n_range))
        p = synth.make_problem(m, n, k=max(3, m // 20), seed=seed * 1000 + i, snr=5.0, dtype=np.float32)
        At = p.At.astype(np.float64)
        alpha, c = 0.7, float(rng.uniform(0.2, 0.8))
        l1, l2 = R.lambdas(At, p.b, alpha, c)
        A, mm = pkg.device_matrix(p.At, pkg.F32)
        x0 = np.zeros(n)
        if warm and i % 3 == 0:
            x0[rng.choice(n, size=3, replace=False)] = rng.normal(size=3)
        x = dev(x0)
        probs.append((At, p.b, l1, l2, x0))
        fits.append((A, mm, dev(p.b), l1, l2, x))
    return probs, fits


@pytest.mark.parametrize("seed,warm", [(1, False), (2, True)])
def test_resident_batch_matches_the_oracle(seed, warm):
    probs, fits = make_fits(48, (20, 400), (200, 6000), seed, warm)
    st, res, info = pkg.ssnal_en_solve_batch_resident(fits)
    assert st == pkg.OK, [r.status for r in res]
    for (At, b, l1, l2, x0), f, r in zip(probs, fits, res):
        assert r.status == pkg.OK and r.kkt1 <= 1e-6 and r.kkt3 <= 1e-6
        ro = R.solve(At, b, l1, l2, x0=x0)
        assert ro.converged
        assert_parity(At, b, l1, l2, f[5].cpu().numpy(), ro)


def test_resident_batch_tuner_does_not_change_results():
    # enough fits for the tuner (three slices of one fit per SM, then the rest)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    probs, fits = make_fits(4 * sms + 40, (10, 60), (50, 400), 5)
    st, res, info = pkg.ssnal_en_solve_batch_resident(fits)
    assert st == pkg.OK and info[0] in (4, 8, 16)
    xs = [f[5].clone() for f in fits]
    # the same fits again, all with one fixed depth: a batch below the tuning size
    for k in range(0, len(fits), sms):
        part = fits[k:k + sms]
        for f, (At, b, l1, l2, x0) in zip(part, probs[k:k + sms]):
            f[5].zero_()
        st2, res2, info2 = pkg.ssnal_en_solve_batch_resident(part)
        assert st2 == pkg.OK
    for x, f in zip(xs, fits):
        np.testing.assert_array_equal(x.cpu().numpy(), f[5].cpu().numpy())
    for (At, b, l1, l2, x0), f in list(zip(probs, fits))[::17]:
        ro = R.solve(At, b, l1, l2)
        assert_parity(At, b, l1, l2, f[5].cpu().numpy(), ro)


def test_resident_batch_hands_hard_fits_to_the_regular_path():
    # duplicated columns, lambda2 = 1e-6, sigma0 = 1e4: the FP32 Newton solve cannot work
    p = synth.make_problem(100, 1000, k=10, seed=5, snr=2)
    At = p.At.copy()
    supp = np.flatnonzero(p.x_true)
    for i in range(5):
        At[999 - i] = At[supp[i]]
    At32 = At.astype(np.float32)
    A64 = At32.astype(np.float64)
    lam1, _ = R.lambdas(A64, p.b, 0.999, 0.2)
    lam2 = 1e-6
    A, mm = pkg.device_matrix(At32, pkg.F32)
    x = torch.zeros(1000, dtype=torch.float64, device="cuda")
    o = pkg.ssnal_en_default_options(sigma0=1e4)
    st, res, info = pkg.ssnal_en_solve_batch_resident([(A, mm, dev(p.b), lam1, lam2, x)], options=o)
    assert st == pkg.OK and info[1] == 1
    ro = R.solve(A64, p.b, lam1, lam2, opts=R.Options(sigma0=1e4))
    assert_parity(A64, p.b, lam1, lam2, x.cpu().numpy(), ro)
