"""The allocation-free entry point ssnal_en_prox_active_static.

It serves callers that may not allocate device memory; its scratch is a fixed
array inside the library.  Checked through the C ABI against the context-based
ssnal_en_op_prox_active (bit-exact: indices and prox values), on two calls in a
row with different sizes, so that the second call cannot lean on anything the
first one left in the shared scratch.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2006_03970_gb300 as pkg  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_03970_gb300 import build
    build.build()
    return pkg.load_library()


def _case(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=n) * (rng.random(n) < 0.3)
    u = rng.normal(size=n) * 3
    return x, u


def _existing(x, u, sigma, l1, l2):
    n = x.size
    ctx = pkg.Context(np.zeros((n, 2)))
    J = torch.zeros(n, dtype=torch.int32, device="cuda")
    wJ = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = pkg.ssnal_en_op_prox_active(ctx.ctx, torch.as_tensor(x, device="cuda"), torch.as_tensor(u, device="cuda"),
                                    sigma, l1, l2, J, wJ)
    ctx.close()
    return r, J[:r].cpu().numpy(), wJ[:r].cpu().numpy()


def test_static_prox_active_matches_context_entry_point(lib):
    cases = [(1_500_007, 11, 0.37, 2.1, 0.8), (4_099, 12, 1.3, 0.4, 0.05)]
    expected = [_existing(*_case(n, seed), s, l1, l2) for n, seed, s, l1, l2 in cases]
    got = []
    for n, seed, s, l1, l2 in cases:  # two calls in a row on the shared scratch
        x, u = _case(n, seed)
        J = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        wJ = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        r = pkg.ssnal_en_prox_active_static(torch.as_tensor(x, device="cuda"), torch.as_tensor(u, device="cuda"),
                                            s, l1, l2, J, wJ)
        got.append((r, J[:r].cpu().numpy(), wJ[:r].cpu().numpy()))
    for (r0, J0, w0), (r1, J1, w1) in zip(expected, got):
        assert r0 == r1 and r0 > 0
        np.testing.assert_array_equal(J1, J0)
        np.testing.assert_array_equal(w1, w0)


def test_static_prox_active_rejects_sizes_beyond_its_scratch(lib):
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    J = torch.zeros(8, dtype=torch.int32, device="cuda")
    r = ctypes.c_int64(-1)
    st = lib.ssnal_en_prox_active_static(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                         pkg.STATIC_MAX_N + 1, 1.0, 1.0, 1.0, ctypes.c_void_p(J.data_ptr()),
                                         ctypes.c_void_p(x.data_ptr()), ctypes.byref(r), None)
    assert st == pkg.ENOTSUP and r.value == -1


@pytest.mark.parametrize("n", [1, 257, 100_003, 2_097_152])
def test_static_prox_active_matches_the_oracle(lib, n):
    # against the definitions themselves (eq. Q_def, eq. prox_elastic): J bit-exact and
    # ascending, w_J with the same rounding sequence as the elementwise definition
    from oracle import ssnal_en_ref as R
    x, u = _case(n, 100 + n)
    sigma, l1, l2 = 0.37, 2.1, 0.8
    J = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    wJ = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    r = pkg.ssnal_en_prox_active_static(torch.as_tensor(x, device="cuda"), torch.as_tensor(u, device="cuda"),
                                        sigma, l1, l2, J, wJ)
    v = x - sigma * u
    Jo = R.active_set(v, sigma, l1)
    assert r == len(Jo)
    np.testing.assert_array_equal(J[:r].cpu().numpy(), Jo)
    np.testing.assert_array_equal(wJ[:r].cpu().numpy(), R.prox_sigma_p(v, sigma, l1, l2)[Jo])


def test_static_prox_active_checks_its_tensors(lib):
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    J = torch.zeros(8, dtype=torch.int32, device="cuda")
    wJ = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):  # J shorter than n
        pkg.ssnal_en_prox_active_static(x, x, 1.0, 1.0, 1.0, J, wJ)
    with pytest.raises(ValueError):  # wrong dtype
        pkg.ssnal_en_prox_active_static(x.float(), x, 1.0, 1.0, 1.0, J, wJ)
