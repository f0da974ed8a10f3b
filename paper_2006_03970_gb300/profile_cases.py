"""Small, self-contained workloads for kernel profiling (ncu) of the hot path.

Each case is sized so that a full metric capture of one kernel ends within a minute
or two while its operands still exceed the 129 MB L2 of a GB300:

  precision-small  the precision workload's generator (50-feature AR(1) blocks, rho 0.5,
                   FP32 generated, standardized, stored BF16) at m = 1000, n = 100000
                   (200 MB), one mixed-form fit per alpha in {0.5, 0.9}, c = 0.3
  newton-730       one Newton direction of the SMW form (eq. smw_formula) at m = 1000,
                   r = 730 (the active-set size of the precision workload at alpha 0.5) on
                   BF16 storage: the BF16 tensor-core SYRK, the cluster Cholesky and the
                   triangular solves with their refinement
  newton-1000      one Newton direction of the m x m form (eq. AJ_system) at m = 1000,
                   r = 1500 on BF16 storage: SYRK over K = r, the super-block Cholesky
                   (cluster factors, block solve, trailing update) and the cluster solves
  prox-1e6         the active-set pass and its compaction at n = 1e6, ~0.1 % active
  batch-152        the device-resident batched solver, 152 instances of the batched
                   workload's generator with n <= 5000 (one launch of k_batch_solve)
  shared-4         four mixed-form fits on the precision-small matrix advanced together
                   (ssnal_en_solve_shared): one merged pass over A per Newton step

    python -m paper_2006_03970_gb300.profile_cases precision-small [newton-730 ...]
"""
from __future__ import annotations

import sys

import numpy as np


def precision_small(n=100_000, m=1000, fits=1):
    import torch
    import paper_2006_03970_gb300 as pkg
    from paper_2006_03970_gb300 import synth
    p = synth.config3(m=m, n=n)
    bits = synth.to_bf16_bits(p.At)
    ctx = pkg.Context(bits, dtype=pkg.BF16, options=pkg.ssnal_en_default_options(precision=1))
    b = torch.as_tensor(p.b, dtype=torch.float64, device="cuda")
    X = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    out = []
    for _ in range(fits):
        for alpha in (0.5, 0.9):
            st, res, done = pkg.ssnal_en_path(ctx.ctx, b, alpha, [0.3], X)
            out.append((alpha, res[0].status, res[0].newton_iters, res[0].active))
    torch.cuda.synchronize()
    ctx.close()
    return out


def newton_730(m=1000, r=730, repeats=3):
    import torch
    import paper_2006_03970_gb300 as pkg
    from paper_2006_03970_gb300 import synth
    rng = np.random.default_rng(730)
    At = rng.normal(size=(r + 64, m)).astype(np.float32)
    bits = synth.to_bf16_bits(At)
    ctx = pkg.Context(bits, dtype=pkg.BF16, options=pkg.ssnal_en_default_options(precision=1))
    J = torch.arange(r, dtype=torch.int32, device="cuda")
    g = torch.as_tensor(rng.normal(size=m), device="cuda")
    gd = torch.empty(m, dtype=torch.float64, device="cuda")
    pkg.ssnal_en_op_grad(ctx.ctx, J, torch.zeros(r, dtype=torch.float64, device="cuda"), r, -g,
                         torch.zeros(m, dtype=torch.float64, device="cuda"), gd)
    d = torch.empty(m, dtype=torch.float64, device="cuda")
    for _ in range(repeats):
        pkg.ssnal_en_op_newton(ctx.ctx, r, 0.5, g, d)
    torch.cuda.synchronize()
    ctx.close()
    return float(d.abs().max())


def newton_1000(m=1000, r=1500, repeats=3):
    """One Newton direction of the m x m form (eq. AJ_system) at m = 1000, r = 1500 (the
    first Newton steps of the precision workload, where r > m): the tensor-core SYRK over
    K = r, the super-block Cholesky (two 512-column cluster factors, the block solve and
    the trailing update) and the cluster triangular solves."""
    return newton_730(m=m, r=r, repeats=repeats)


def prox_1e6(n=1_000_000, m=64, repeats=3):
    """The active-set pass (eq. Q_def, eq. prox_elastic) and its ordered compaction at
    n = 1e6 with about 0.1 % of the columns active (the precision workload's r ~ 730)."""
    import torch
    import paper_2006_03970_gb300 as pkg
    rng = np.random.default_rng(6)
    bits = np.zeros((n, m), dtype=np.uint16)
    ctx = pkg.Context(bits, dtype=pkg.BF16, options=pkg.ssnal_en_default_options(precision=1))
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    u = torch.as_tensor(rng.normal(size=n), device="cuda")
    J = torch.empty(n, dtype=torch.int32, device="cuda")
    wJ = torch.empty(n, dtype=torch.float64, device="cuda")
    r = 0
    for _ in range(repeats):
        r = pkg.ssnal_en_op_prox_active(ctx.ctx, x, u, 1.0, 3.3, 0.1, J, wJ)
    torch.cuda.synchronize()
    ctx.close()
    return r


def batch_152(count=152):
    """The device-resident batched solver on one instance per SM: the batched workload's
    generator (m log-uniform [50, 500], n log-uniform [1e3, 5e4], FP32) with n capped at
    5000, so that one launch of k_batch_solve runs a few milliseconds."""
    import torch
    import paper_2006_03970_gb300 as pkg
    from paper_2006_03970_gb300 import synth
    probs = [p for p in synth.config4_instances(4 * count) if p.At.shape[0] <= 5000][:count]
    fits, keep = [], []
    for p in probs:
        A = torch.as_tensor(np.ascontiguousarray(p.At, dtype=np.float32), device="cuda")
        b = torch.as_tensor(p.b, dtype=torch.float64, device="cuda")
        x = torch.zeros(p.At.shape[0], dtype=torch.float64, device="cuda")
        g = float(np.abs(p.At.astype(np.float64) @ p.b).max())
        fits.append((A, p.At.shape[1], b, p.c * g, (1 - p.alpha) / p.alpha * p.c * g, x))
        keep.append(A)
    st, res, info = pkg.ssnal_en_solve_batch_resident(fits)
    torch.cuda.synchronize()
    return st, sum(1 for r in res if r.status == 0), info


def shared_4(n=100_000, m=1000):
    """Four mixed-form fits on the precision-small matrix through ssnal_en_solve_shared: their
    Newton-step passes over A merged into one k_stream_multi launch per step."""
    import torch
    import paper_2006_03970_gb300 as pkg
    from paper_2006_03970_gb300 import synth
    p = synth.config3(m=m, n=n)
    bits = synth.to_bf16_bits(p.At)
    opts = pkg.ssnal_en_default_options(precision=1)
    A, mm = pkg.device_matrix(bits, pkg.BF16)
    ctxs = [pkg.Context(A, m=mm, dtype=pkg.BF16, options=opts) for _ in range(4)]
    rng = np.random.default_rng(4)
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    inst = []
    for i, c in enumerate(ctxs):
        b = torch.as_tensor(p.b + 0.1 * rng.standard_normal(m), device="cuda")
        pkg.ssnal_en_op_at_y(c.ctx, b, u)
        g = u.abs().max().item()
        inst.append((c.ctx, b, 0.3 * g, 0.3 * g, torch.zeros(n, dtype=torch.float64, device="cuda"), None))
    st, res, passes = pkg.ssnal_en_solve_shared(inst)
    torch.cuda.synchronize()
    for c in ctxs:
        c.close()
    return st, [r.newton_iters for r in res], passes


CASES = {"precision-small": precision_small, "newton-730": newton_730, "newton-1000": newton_1000,
         "shared-4": shared_4, "prox-1e6": prox_1e6, "batch-152": batch_152}


def main(argv):
    if not argv or any(a not in CASES for a in argv):
        print(__doc__)
        return 2
    import paper_2006_03970_gb300 as pkg
    pkg.load_library()
    for a in argv:
        print(a, CASES[a]())
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
