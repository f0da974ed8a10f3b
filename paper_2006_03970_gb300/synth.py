"""Seeded synthetic Elastic Net workloads (inputs only; no solver arithmetic).

The paper's simulation design (Sec. 4.1) draws a standard-normal design matrix,
a sparse true coefficient vector x_t and b = A x_t + eps with a fixed
signal-to-noise ratio snr = var(A x_t) / s_eps^2.  The workloads below follow
that recipe with the variations of the benchmark configurations: block
Toeplitz (AR(1)) feature correlation, random-sign uniform magnitudes for the
nonzeros, and standardized columns (mean 0, population variance 1).

Storage convention: the design matrix is returned as ``At`` with shape (n, m),
C-contiguous, i.e. ``At[j]`` is feature column j of A.  This is exactly the
column-major m x n layout the CUDA path streams.

This module holds no part of the solver: it neither thresholds nor solves.  It
is the one module shared by the oracle-side tests and the CUDA-side tests and
benchmarks, so both see bit-identical inputs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem", "make_problem", "config1", "config2", "config3", "config4_instances",
    "genotype_matrix", "path_grid", "to_bf16_bits", "bf16_bits_to_f32",
]


@dataclasses.dataclass
class Problem:
    At: np.ndarray          # (n, m) feature-major == column-major A
    b: np.ndarray           # (m,) float64
    x_true: np.ndarray      # (n,) float64
    alpha: float
    c: float | None = None
    seed: int = 0

    @property
    def m(self) -> int:
        return self.At.shape[1]

    @property
    def n(self) -> int:
        return self.At.shape[0]


def _design(rng, m, n, block, rho, dtype):
    """Rows ~ N(0, Sigma), Sigma block diagonal with rho^|i-j| inside blocks.

    Within a block of consecutive features the AR(1) recursion
    f_0 = e_0, f_k = rho f_{k-1} + sqrt(1-rho^2) e_k gives unit variances and
    Cov(f_i, f_j) = rho^|i-j| exactly; blocks are independent.
    """
    At = rng.standard_normal((n, m), dtype=np.float32 if dtype == np.float32 else np.float64)
    if block > 1 and rho != 0.0:
        c = math.sqrt(1.0 - rho * rho)
        for start in range(0, n, block):
            stop = min(start + block, n)
            # recursion along the feature index inside the block
            for k in range(start + 1, stop):
                At[k] *= c
                At[k] += rho * At[k - 1]
    return At


def _standardize(At):
    """Centre each column to mean 0 and scale to population variance 1."""
    mu = At.mean(axis=1, keepdims=True, dtype=np.float64)
    At -= mu.astype(At.dtype)
    sd = np.sqrt((At.astype(np.float64) ** 2).mean(axis=1, keepdims=True)) if At.dtype == np.float64 \
        else np.sqrt(np.einsum("ij,ij->i", At, At, dtype=np.float64)[:, None] / At.shape[1])
    sd[sd == 0] = 1.0
    At /= sd.astype(At.dtype)
    return At


def _sparse_truth(rng, n, k, lo, hi):
    x = np.zeros(n)
    idx = rng.choice(n, size=k, replace=False)
    sign = rng.choice(np.array([-1.0, 1.0]), size=k)
    x[idx] = sign * rng.uniform(lo, hi, size=k)
    return x


def _response(rng, At, x, snr):
    """b = A x + eps, eps ~ N(0, s^2) with s^2 = var(A x) / snr (population var)."""
    supp = np.flatnonzero(x)
    Ax = At[supp].astype(np.float64).T @ x[supp]
    s = math.sqrt(Ax.var() / snr) if snr > 0 else 0.0
    return Ax + s * rng.standard_normal(At.shape[1])


def make_problem(m, n, *, k, lo=1.0, hi=3.0, snr=5.0, alpha=0.8, c=None, block=1, rho=0.0,
                 seed=0, dtype=np.float64) -> Problem:
    """Generic generator: the paper's simulation recipe with the knobs above."""
    rng = np.random.Generator(np.random.PCG64(seed))
    At = _standardize(_design(rng, m, n, block, rho, dtype))
    x = _sparse_truth(rng, n, min(k, n), lo, hi)
    b = _response(rng, At, x, snr)
    return Problem(At=At, b=b, x_true=x, alpha=alpha, c=c, seed=seed)


def config1(seed=0) -> Problem:
    """One FP64 fit: m=100, n=2000, iid N(0,1), 10 nonzeros +-U[1,3], snr 5, alpha .8, c .5."""
    return make_problem(100, 2000, k=10, snr=5.0, alpha=0.8, c=0.5, seed=seed)


def path_grid(K=20, c_min=0.05):
    """Geometric grid from 1.0 down to c_min (K points), descending."""
    return np.array([c_min ** (k / (K - 1)) for k in range(K)]) if K > 1 else np.array([1.0])


def config2(seed=2, m=500, n=100_000) -> Problem:
    """FP64 path workload: m=500, n=1e5, 100-feature AR(1) blocks rho .7, 20 nonzeros, alpha .6."""
    return make_problem(m, n, k=20, snr=5.0, alpha=0.6, block=100, rho=0.7, seed=seed)


def config3(seed=3, m=1000, n=1_000_000, alpha=0.5) -> Problem:
    """Precision workload: m=1000, n=1e6, 50-feature blocks rho .5, generated FP32, 50 nonzeros, snr 3, c .3."""
    return make_problem(m, n, k=50, snr=3.0, alpha=alpha, c=0.3, block=50, rho=0.5, seed=seed,
                        dtype=np.float32)


def config4_instances(count=512, seed=4):
    """Uneven batch: m log-uniform [50,500], n log-uniform [1e3,5e4], alpha .7, c ~ U[.2,.8]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ms = np.rint(np.exp(rng.uniform(math.log(50), math.log(500), count))).astype(int)
    ns = np.rint(np.exp(rng.uniform(math.log(1e3), math.log(5e4), count))).astype(int)
    cs = rng.uniform(0.2, 0.8, count)
    out = []
    for i in range(count):
        p = make_problem(int(ms[i]), int(ns[i]), k=max(5, int(ms[i]) // 20), snr=5.0, alpha=0.7,
                         c=float(cs[i]), seed=seed * 1_000_000 + i, dtype=np.float32)
        out.append(p)
    return out


def genotype_matrix(m, n, seed=5):
    """int8 codes {0,1,2} ~ Binomial(2, p_j), p_j ~ U(0.05, 0.5), plus per-column mean/scale.

    Returns (codes (n, m) int8 feature-major, mean (n,) float32, scale (n,) float32) where the
    standardized entry is (code - mean) * scale; scale is 0 for a constant column.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    p = rng.uniform(0.05, 0.5, n)
    codes = rng.binomial(2, p[:, None], size=(n, m)).astype(np.int8)
    mean = codes.mean(axis=1, dtype=np.float64)
    var = (codes.astype(np.float64) ** 2).mean(axis=1) - mean ** 2
    scale = np.where(var > 0, 1.0 / np.sqrt(np.maximum(var, 1e-300)), 0.0)
    return codes, mean.astype(np.float32), scale.astype(np.float32)


def to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest-even); returns the uint16 bit patterns."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    rounding = ((u >> 16) & 1) + 0x7FFF
    return ((u + rounding) >> 16).astype(np.uint16)


def bf16_bits_to_f32(h: np.ndarray) -> np.ndarray:
    return (h.astype(np.uint32) << 16).view(np.float32)
