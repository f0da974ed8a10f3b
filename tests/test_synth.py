"""The seeded input generators follow the stated recipe (Sec. 4.1 design plus the AR(1) blocks,
standardized columns, signed uniform nonzeros and the signal-to-noise ratio), are
deterministic, and round to BF16 like PyTorch does."""
import numpy as np
import pytest

from paper_2006_03970_gb300 import synth


def test_standardized_columns_and_shapes():
    p = synth.make_problem(200, 300, k=7, seed=1, block=10, rho=0.6)
    assert p.At.shape == (300, 200) and p.At.flags["C_CONTIGUOUS"] and p.b.shape == (200,)
    np.testing.assert_allclose(p.At.mean(axis=1), 0.0, atol=1e-12)
    np.testing.assert_allclose((p.At ** 2).mean(axis=1), 1.0, rtol=1e-12)


def test_ar1_blocks():
    # neighbours inside a block correlate at rho, features of different blocks do not
    rho, block = 0.7, 10
    p = synth.make_problem(20000, 40, k=3, seed=2, block=block, rho=rho)
    corr = p.At @ p.At.T / p.At.shape[1]  # unit population variance after standardizing
    inside = [corr[j, j + 1] for j in range(39) if (j + 1) % block != 0]
    across = [corr[j, j + 1] for j in range(39) if (j + 1) % block == 0]
    assert abs(np.mean(inside) - rho) < 0.02
    assert abs(np.mean(corr[0, 2:block]) - np.mean([rho ** d for d in range(2, block)])) < 0.03
    assert max(abs(c) for c in across) < 0.05


def test_sparse_truth_and_snr():
    p = synth.make_problem(4000, 500, k=20, lo=1.0, hi=3.0, snr=5.0, seed=3)
    nz = np.flatnonzero(p.x_true)
    assert nz.size == 20
    mags = np.abs(p.x_true[nz])
    assert np.all((mags >= 1.0) & (mags <= 3.0))
    assert 0 < np.count_nonzero(p.x_true > 0) < 20  # both signs occur
    signal = p.At.T @ p.x_true
    noise = p.b - signal
    assert signal.var() / noise.var() == pytest.approx(5.0, rel=0.08)


def test_deterministic_by_seed():
    a = synth.make_problem(50, 80, k=5, seed=11, block=8, rho=0.5)
    b = synth.make_problem(50, 80, k=5, seed=11, block=8, rho=0.5)
    c = synth.make_problem(50, 80, k=5, seed=12, block=8, rho=0.5)
    assert np.array_equal(a.At, b.At) and np.array_equal(a.b, b.b) and np.array_equal(a.x_true, b.x_true)
    assert not np.array_equal(a.At, c.At)


def test_fp32_generation():
    p = synth.make_problem(64, 100, k=4, seed=5, dtype=np.float32, block=5, rho=0.5)
    assert p.At.dtype == np.float32 and p.b.dtype == np.float64
    np.testing.assert_allclose((p.At.astype(np.float64) ** 2).mean(axis=1), 1.0, rtol=1e-5)


def test_path_grid_geometric_descending():
    g = synth.path_grid(20, 0.05)
    assert g.size == 20 and g[0] == 1.0 and g[-1] == pytest.approx(0.05, rel=1e-14)
    ratios = g[1:] / g[:-1]
    np.testing.assert_allclose(ratios, ratios[0], rtol=1e-12)
    assert np.all(np.diff(g) < 0)
    assert synth.path_grid(1).tolist() == [1.0]


def test_batch_instances_ranges():
    inst = synth.config4_instances(count=40, seed=4)
    ms = np.array([p.m for p in inst])
    ns = np.array([p.n for p in inst])
    assert ms.min() >= 50 and ms.max() <= 500 and ns.min() >= 1000 and ns.max() <= 50000
    assert all(p.At.dtype == np.float32 and 0.2 <= p.c <= 0.8 and p.alpha == 0.7 for p in inst)


def test_genotype_codes_and_standardization():
    codes, mean, scale = synth.genotype_matrix(500, 64, seed=5)
    assert codes.dtype == np.int8 and set(np.unique(codes)) <= {0, 1, 2}
    std = (codes.astype(np.float64) - mean[:, None]) * scale[:, None]
    live = scale > 0
    np.testing.assert_allclose(std[live].mean(axis=1), 0.0, atol=1e-6)
    np.testing.assert_allclose((std[live] ** 2).mean(axis=1), 1.0, rtol=1e-5)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    a = np.concatenate([rng.normal(size=4000).astype(np.float32),
                        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, -0.0, 3.0e38], np.float32)])
    ours = synth.bf16_bits_to_f32(synth.to_bf16_bits(a))
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert ours[4000] == 1.0 and ours[4001] == np.float32(1 + 2 ** -6)
