#!/usr/bin/env python
"""Benchmark of the SsNAL-EN hot path on GB300.

Workload (one "step"): the FP64 warm-started regularization path on the
synthetic design of the path configuration -- m = 500 observations,
n = 100,000 features in 100-feature AR(1) blocks (rho = 0.7), 20 nonzeros of
+-U[1,3], snr 5, alpha = 0.6, c = 1.0 -> 0.05 geometric (20 points), KKT
tolerance 1e-6.  The metric is Elastic Net fits per second, counting a fit
only when both res(kkt1) and res(kkt3) (FP64) are <= 1e-6.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle on the same workload (host cores).
For N > 1 (torchrun) every rank solves its own replica of the workload
(independent problems, no data-path collective); value = all fits / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

STREAM_TRAFFIC_BYTES = 401668352 + 3752704  # ncu, one k_stream_lane<kModeT> launch, m=500 n=1e5
METRIC = "EN fits/s to KKT<=1e-6"
UNIT = "fits/s"
WORKLOAD = ("FP64 warm-started Elastic Net path: m=500, n=100000, 100-feature AR(1) blocks rho=0.7, "
            "20 nonzeros +-U[1,3], snr 5, alpha=0.6, c 1.0->0.05 geometric (20 points), tol 1e-6, seed 2")
M, N_FEAT, K_POINTS, ALPHA, SEED = 500, 100_000, 20, 0.6, 2
TOL = 1e-6


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(elapsed, units, device):
    """(max of `elapsed`, sum of `units`) over the ranks of the default process group;
    the inputs unchanged without one.  The job's time is its slowest rank's; every rank
    contributes the fits it completed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return elapsed, units
    t = torch.tensor([float(elapsed), float(units)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return tmax[0].item(), t[1].item()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clocks and throttle reasons during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < len(self.FIELDS):
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx = float(parts[1])
                except ValueError:
                    continue
                for name, val in zip(self.NAMES, parts[3:7]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _workload():
    from paper_2006_03970_gb300 import synth
    p = synth.config2(seed=SEED, m=M, n=N_FEAT)
    return p, list(synth.path_grid(K_POINTS, 0.05))


def _count_fits(results, done):
    return sum(1 for r in results[:done] if r.status == 0 and r.kkt1 <= TOL and r.kkt3 <= TOL)


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import ssnal_en_ref as R
    p, grid = _workload()
    At = np.ascontiguousarray(p.At, dtype=np.float64)
    for _ in range(args.warmup):
        R.path(At, p.b, ALPHA, grid)
    fits, t0 = 0, time.perf_counter()
    for _ in range(args.steps):
        res = R.path(At, p.b, ALPHA, grid)
        fits += sum(1 for r in res if r.converged and r.kkt1 <= TOL and r.kkt3 <= TOL)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    value = fits / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "inputs larger than L2 (A is 400 MB)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full 20-point paths (NumPy/SciPy FP64, default BLAS threads)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline():
    """The FP64 oracle on a bounded sample: one full 20-point path of the same workload."""
    import numpy as np
    from oracle import ssnal_en_ref as R
    p, grid = _workload()
    At = np.ascontiguousarray(p.At, dtype=np.float64)
    t0 = time.perf_counter()
    res = R.path(At, p.b, ALPHA, grid)
    dt = time.perf_counter() - t0
    fits = sum(1 for r in res if r.converged and r.kkt1 <= TOL and r.kkt3 <= TOL)
    return {"value": fits / dt, "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": "one full 20-point path of the same workload (NumPy/SciPy FP64, default BLAS threads)",
            "seconds": dt}


def run_gpu(args):
    import numpy as np
    import torch

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2006_03970_gb300 as pkg
    pkg.load_library()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    p, grid = _workload()
    ctx = pkg.Context(p.At)
    b = torch.as_tensor(p.b, dtype=torch.float64, device="cuda")
    X = torch.zeros((len(grid), ctx.n), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        pkg.ssnal_en_path(ctx.ctx, b, ALPHA, grid, X)
    torch.cuda.synchronize()
    barrier()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)  # let the sampler start before the timed region
    prof0 = pkg.ssnal_en_profile(ctx.ctx, True, True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fits = 0
    newton = 0  # one A^T d stream launch per Newton step
    for _ in range(args.steps):
        st, res, done = pkg.ssnal_en_path(ctx.ctx, b, ALPHA, grid, X)
        fits += _count_fits(res, done)
        newton += sum(r.newton_iters for r in res[:done])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    prof1 = pkg.ssnal_en_profile(ctx.ctx, False, False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms, fits_all = reduce_over_ranks(ms, fits, "cuda")
    value = fits_all / (ms / 1e3)

    # end to end through the public C ABI with host buffers (b in, all solutions out)
    b_host = torch.empty(M, dtype=torch.float64, pin_memory=True)
    b_host.copy_(torch.from_numpy(p.b))
    X_host = torch.empty((len(grid), ctx.n), dtype=torch.float64, pin_memory=True)
    bh, xh = b_host.numpy(), X_host.numpy()
    pkg.ssnal_en_path_host(ctx.ctx, bh, ALPHA, grid, xh)
    barrier()
    t0 = time.perf_counter()
    efits = 0
    for _ in range(args.steps):
        st, res, done = pkg.ssnal_en_path_host(ctx.ctx, bh, ALPHA, grid, xh)
        efits += _count_fits(res, done)
    edt = time.perf_counter() - t0
    barrier()
    edt, efits = reduce_over_ranks(edt, efits, "cuda")
    e2e_value = efits / edt

    peak, peak_kind = _peaks()
    launches = prof1["stream_launches"] - 0
    s_ms = prof1["stream_ms"]
    achieved = (prof1["stream_bytes"] / (s_ms / 1e3) / 1e9) if s_ms > 0 else None
    roofline = {"kernel": "k_stream_lane<kModeT> (t = A^T d over the pre-split float pair copy, "
                          "fused line-search trial sums)",
                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                # dram__bytes_read.sum + dram__bytes_write.sum of one launch of this kernel on this
                # workload (profiles/k_stream_lane_modeT_m500_n1e5.md)
                "traffic": STREAM_TRAFFIC_BYTES, "traffic_unit": "bytes per launch",
                "peak_kind": peak_kind, "launches": newton, "timed_launches": launches,
                "timed_every": 8,
                "avg_launch_us": (s_ms / launches * 1e3) if launches else None,
                "bytes_per_launch": (prof1["stream_bytes"] / launches) if launches else None,
                "share_of_step": (s_ms / launches * newton / ms) if (ms > 0 and launches) else None}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "inputs larger than L2 (A is 400 MB, L2 129 MB)",
                       "fits_per_step": K_POINTS, "parallelism": "replicas" if world > 1 else "single GPU"},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * M,
                    "d2h_bytes_per_step": 8 * len(grid) * ctx.n},
            "gpu_launches": prof1["kernel_launches"] - prof0["kernel_launches"],
            "roofline": roofline}
    if rank == 0 and world == 1 and not args.no_mixed:
        line["mixed_vs_fp64"] = mixed_vs_fp64()
    if rank == 0 and world == 1 and not args.no_batch:
        line["batched"] = batched_fits()
    if rank == 0 and world == 1 and not args.no_serve:
        line["serving"] = serve_workload(args.serve_requests, args.serve_matrices)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def mixed_vs_fp64(steps=3):
    """The precision configuration on one GPU: m=1000, n=1e6, 50-feature AR(1) blocks (rho 0.5),
    generated in FP32 and standardized; 50 nonzeros +-U[1,3], snr 3, c = 0.3, alpha in {0.5, 0.9}.
    The mixed form stores A as BF16 (2 GB; FP32-accumulated Newton passes, float-float refresh of
    u = A^T y before each stopping test); the FP64 form stores the FP32 values as FP64 (8 GB).
    Reported: fits/s of each form (CUDA events, inputs resident), the mixed/FP64 ratio, the
    storage+solver error of the mixed solution against the FP64 path's, and the achieved GB/s of
    the mixed Newton pass."""
    import numpy as np
    import torch
    import paper_2006_03970_gb300 as pkg
    from paper_2006_03970_gb300 import synth
    p = synth.config3()
    bits = synth.to_bf16_bits(p.At)
    ctx_m = pkg.Context(bits, dtype=pkg.BF16, options=pkg.ssnal_en_default_options(precision=1))
    ctx_f = pkg.Context(p.At.astype(np.float64))
    b = torch.as_tensor(p.b, dtype=torch.float64, device="cuda")
    grid = np.array([0.3])
    out = {"workload": "m=1000, n=1000000, 50-feature AR(1) blocks rho=0.5, FP32 generated and "
                       "standardized, 50 nonzeros +-U[1,3], snr 3, c=0.3, seed 3",
           "mixed": "A in BF16 (2 GB), FP32-accumulated Newton passes, float-float u refresh, "
                    "BF16 tensor-core SYRK, FP32 Cholesky + FP64 refinement, FP64 KKT",
           "fp64": "A in FP64 (8 GB), float-float passes over the pre-split copy",
           "cases": []}
    stream = torch.cuda.current_stream()
    for alpha in (0.5, 0.9):
        case = {"alpha": alpha}
        xs = {}
        for name, ctx in (("mixed", ctx_m), ("fp64", ctx_f)):
            X = torch.zeros((1, ctx.n), dtype=torch.float64, device="cuda")
            pkg.ssnal_en_path(ctx.ctx, b, alpha, grid, X)
            torch.cuda.synchronize()
            pkg.ssnal_en_profile(ctx.ctx, True, True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ok = 0
            for _ in range(steps):
                st, res, done = pkg.ssnal_en_path(ctx.ctx, b, alpha, grid, X)
                ok += _count_fits(res, done)
            e1.record(stream)
            torch.cuda.synchronize()
            prof = pkg.ssnal_en_profile(ctx.ctx, False, False)
            ms = e0.elapsed_time(e1) / steps
            r = res[0]
            case[name] = {"fits_per_s": (ok / steps) / (ms / 1e3), "ms_per_fit": ms, "kkt1": r.kkt1,
                          "kkt3": r.kkt3, "al_iters": r.al_iters, "newton_iters": r.newton_iters,
                          "active": r.active,
                          "stream_gbs": (prof["stream_bytes"] / (prof["stream_ms"] / 1e3) / 1e9)
                          if prof["stream_ms"] > 0 else None}
            xs[name] = X[0].cpu().numpy()
        case["mixed_over_fp64"] = case["mixed"]["fits_per_s"] / case["fp64"]["fits_per_s"]
        xm, xf = xs["mixed"], xs["fp64"]
        case["x_rel_err_mixed_vs_fp64"] = float(np.abs(xm - xf).max() / max(np.abs(xf).max(), 1e-300))
        case["support_mixed_fp64"] = [int(np.count_nonzero(xm)), int(np.count_nonzero(xf))]
        out["cases"].append(case)
    ctx_m.close()
    ctx_f.close()
    return out


def batched_fits(count=512):
    """The batched configuration: 512 independent fits, m log-uniform in [50, 500], n log-uniform in
    [1e3, 5e4], A iid N(0,1) standardized and stored in FP32, max(5, m/20) nonzeros, snr 5,
    alpha 0.7, c ~ U[0.2, 0.8] (seed 4).  All matrices are resident; each timed batch starts from
    x = 0.  Reported: fits/s of ssnal_en_solve_batch (tuned worker count) and, for comparison,
    of the same instances solved one after another."""
    import numpy as np
    import torch
    import paper_2006_03970_gb300 as pkg
    from paper_2006_03970_gb300 import synth
    probs = synth.config4_instances(count)
    ctxs, bs, xs, lams = [], [], [], []
    for p in probs:
        ctxs.append(pkg.Context(p.At, dtype=pkg.F32))
        aty = np.abs(p.At.astype(np.float64) @ p.b).max()
        lams.append((p.alpha * p.c * aty / p.alpha, (1 - p.alpha) / p.alpha * p.c * aty))
        bs.append(torch.as_tensor(p.b, dtype=torch.float64, device="cuda"))
        xs.append(torch.zeros(p.At.shape[0], dtype=torch.float64, device="cuda"))
    inst = [(c.ctx, b, l1, l2, x, None) for c, b, (l1, l2), x in zip(ctxs, bs, lams, xs)]

    def reset():
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()

    reset()
    pkg.ssnal_en_solve_batch(inst, 0)  # warm-up (and tuning)
    reset()
    t0 = time.perf_counter()
    st, res, used = pkg.ssnal_en_solve_batch(inst, 0)
    dt = time.perf_counter() - t0
    ok = sum(1 for r in res if r.status == 0 and r.kkt1 <= TOL and r.kkt3 <= TOL)
    reset()
    t0 = time.perf_counter()
    for c, b, (l1, l2), x in zip(ctxs, bs, lams, xs):
        pkg.ssnal_en_solve(c.ctx, b, l1, l2, x)
    dts = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    mn = sum(p.At.shape[0] * p.At.shape[1] for p in probs)
    return {"workload": f"{count} independent fits, m log-uniform [50,500], n log-uniform [1e3,5e4], FP32 "
                        f"storage ({mn * 4 / 1e9:.2f} GB), alpha 0.7, c ~ U[0.2,0.8], seed 4",
            "fits_per_s": ok / dt, "seconds": dt, "converged": ok, "workers": used,
            "sequential_fits_per_s": count / dts}


def serve_workload(per_rate=400, n_small=16, workers=16, seed=5):
    """The serving configuration: a resident genotype-like A (m=2000, n=500000 int8 codes
    ~ Binomial(2, p_j), p_j ~ U(0.05, 0.5), standardized on the fly by per-column FP32 mean and
    scale) plus `n_small` resident FP32 matrices from the precision workload's generator (m
    log-uniform in [200, 1000], n log-uniform in [1e4, 2e5], 50-feature blocks rho 0.5).  Each
    request: its own x* (30 nonzeros +-U[0.5, 2]), b = A x* + noise at snr 2, alpha ~ U[0.5, 1),
    c ~ U[0.1, 0.8]; its matrix is the genotype one with probability 1/2, else uniform over the
    others.  The server runs the mixed form (precision 1) with `workers` worker streams.  First a
    burst of `per_rate` requests gives the saturation throughput; then Poisson arrivals at
    {0.25, 0.5, 0.75, 0.9, 1.1} x that rate, `per_rate` requests each, give latency percentiles
    (submission to completion, host transfers included)."""
    import math
    import numpy as np
    import torch
    import paper_2006_03970_gb300 as pkg
    from paper_2006_03970_gb300 import synth
    rng = np.random.Generator(np.random.PCG64(seed))
    codes, mean, scale = synth.genotype_matrix(2000, 500_000, seed=seed)
    Ag, mg = pkg.device_matrix(codes, pkg.I8_GENO)
    mats = [(Ag, mg, pkg.I8_GENO, torch.as_tensor(mean, device="cuda"), torch.as_tensor(scale, device="cuda"))]
    host_cols = [lambda idx: (codes[idx].astype(np.float64) - mean[idx, None]) * scale[idx, None]]
    sizes = [(2000, 500_000)]
    for k in range(n_small):
        m = int(round(math.exp(rng.uniform(math.log(200), math.log(1000)))))
        n = int(round(math.exp(rng.uniform(math.log(1e4), math.log(2e5)))))
        q = synth.make_problem(m, n, k=1, seed=seed * 1_000_000 + k, block=50, rho=0.5, dtype=np.float32)
        A, mm = pkg.device_matrix(q.At, pkg.F32)
        mats.append((A, mm, pkg.F32, None, None))
        At = q.At
        host_cols.append(lambda idx, At=At: At[idx].astype(np.float64))
        sizes.append((m, n))

    def request():
        k = 0 if rng.uniform() < 0.5 else int(rng.integers(1, len(mats)))
        m, n = sizes[k]
        idx = rng.choice(n, size=30, replace=False)
        xs = rng.choice([-1.0, 1.0], size=30) * rng.uniform(0.5, 2.0, size=30)
        ax = host_cols[k](idx).T @ xs
        b = ax + math.sqrt(ax.var() / 2.0) * rng.standard_normal(m)
        return k, b, float(rng.uniform(0.5, 1.0)), float(rng.uniform(0.1, 0.8))

    srv = pkg.Server(mats, workers=workers, options=pkg.ssnal_en_default_options(precision=1))

    def run(reqs, arrivals=None):
        t0 = time.perf_counter()
        tickets = []
        for i, (k, b, alpha, c) in enumerate(reqs):
            if arrivals is not None:
                wait = t0 + arrivals[i] - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
            tickets.append((srv.submit_scaled(k, b, alpha, c), k))
        got = [srv.poll(t, k, wait=True) for t, k in tickets]
        lat = np.array([g[2][2] - g[2][0] for g in got])
        span = max(g[2][2] for g in got) - min(g[2][0] for g in got)
        ok = sum(1 for g in got if g[1].status == 0 and g[1].kkt1 <= TOL and g[1].kkt3 <= TOL)
        return {"requests": len(reqs), "converged": ok, "fits_per_s": ok / span,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3)}

    run([request() for _ in range(min(per_rate, 64))])  # warm-up: worker contexts
    burst = run([request() for _ in range(per_rate)])
    sat = burst["fits_per_s"]
    sweep = []
    for f in (0.25, 0.5, 0.75, 0.9, 1.1):
        reqs = [request() for _ in range(per_rate)]
        arrivals = np.cumsum(rng.exponential(1.0 / (f * sat), size=per_rate))
        r = run(reqs, arrivals)
        r["offered_fraction_of_saturation"] = f
        sweep.append(r)
    srv.close()
    return {"workload": f"resident genotype A 2000x500000 int8 (1 GB) + {n_small} FP32 matrices "
                        f"(m in [200,1000], n in [1e4,2e5]); requests 50% genotype, alpha ~ U[0.5,1), "
                        f"c ~ U[0.1,0.8], x* 30 nonzeros, snr 2; mixed form, {workers} worker streams",
            "saturation": burst, "poisson_sweep": sweep}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the BF16-vs-FP64 precision comparison")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--serve-requests", type=int, default=400, help="requests per arrival rate (serving)")
    ap.add_argument("--serve-matrices", type=int, default=16, help="resident FP32 matrices (serving)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
