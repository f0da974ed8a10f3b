#!/usr/bin/env python
"""Benchmark of the SsNAL-EN hot path on GB300.

Headline workload (one "step" = one fit per alpha): the precision configuration --
m = 1000 observations, n = 1,000,000 features in 50-feature AR(1) blocks (rho = 0.5),
generated in FP32, standardized, stored as BF16 (2 GB); 50 nonzeros of +-U[1,3], snr 3,
c = 0.3, alpha in {0.5, 0.9}, KKT tolerance 1e-6 -- solved in the mixed form
(FP32-accumulated Newton passes over the BF16 values, float-float u = A^T y passes,
BF16 tensor-core SYRK, FP32 factor with FP64 refinement and the FP64 system as fallback,
FP64 KKT).  The metric is Elastic Net fits per second, counting a fit only when both
res(kkt1) and res(kkt3) (FP64) are <= 1e-6; the same workload in the FP64 form (A stored
as FP64, 8 GB) is timed beside it ("fp64_form") for the mixed-vs-FP64 comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle on the same workload (host cores).
For N > 1 (torchrun) every rank solves its own replica of the workload
(independent problems, no data-path collective); value = all fits / max time.
Also reported (rank 0, N = 1): the error of both forms against the FP64 oracle, the
FP64 regularization path of the path configuration, the batched and serving workloads.
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

METRIC = "EN fits/s to KKT<=1e-6, mixed vs FP64 on GB300"
UNIT = "fits/s"
TOL = 1e-6
# headline: the precision configuration
M3, N3, C3, ALPHAS3, SEED3 = 1000, 1_000_000, 0.3, (0.5, 0.9), 3
WORKLOAD = ("precision configuration: m=1000, n=1000000, 50-feature AR(1) blocks rho=0.5, generated FP32, "
            "standardized, stored BF16 (2 GB); 50 nonzeros +-U[1,3], snr 3, c=0.3, alpha in {0.5, 0.9} (one fit "
            "each per step), tol 1e-6, seed 3; mixed form")
# secondary: the FP64 regularization path
M2, N2, K2, ALPHA2, SEED2 = 500, 100_000, 20, 0.6, 2
WORKLOAD2 = ("FP64 warm-started Elastic Net path: m=500, n=100000, 100-feature AR(1) blocks rho=0.7, "
             "20 nonzeros +-U[1,3], snr 5, alpha=0.6, c 1.0->0.05 geometric (20 points), tol 1e-6, seed 2")
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch from ncu captures of the
# current kernels.  The pre-split FP64 Newton pass is captured at the path's own size; the
# BF16 passes at n = 1e5 (profiling case precision-small) and scaled to n = 1e6 by the columns
# processed (the per-launch m-vector reads are under 1 %).
TRAFFIC = {
    "split_modeT_m500_n1e5": 405469312,
    "bf16_modeT_m1000_n1e6": 205587712 * 10,
    "bf16ff_modeU_m1000_n1e6": 204056448 * 10,
}


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


def _count_fits(results, done):
    return sum(1 for r in results[:done] if r.status == 0 and r.kkt1 <= TOL and r.kkt3 <= TOL)


def _cores():
    return len(os.sched_getaffinity(0))


def precision_problem():
    """The precision configuration: (problem with FP32 At, BF16 bit patterns of At)."""
    from paper_2006_03970_gb300 import synth
    p = synth.config3(seed=SEED3, m=M3, n=N3)
    return p, synth.to_bf16_bits(p.At)


def _bf16_as_f64(bits):
    import numpy as np
    from paper_2006_03970_gb300 import synth
    return np.ascontiguousarray(synth.bf16_bits_to_f32(bits), dtype=np.float64)


def run_reference(args):
    """The FP64 oracle on the headline workload, on the host cores: each step is one fit
    (alpha alternating 0.5, 0.9) on the stored BF16 values upcast to FP64 -- the problem the
    mixed form solves."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from oracle import blas
    from oracle import ssnal_en_ref as R
    p, bits = precision_problem()
    Ab = _bf16_as_f64(bits)
    del bits
    cores = _cores()
    blas.set_blas_threads(cores)
    lams = {a: R.lambdas(Ab, p.b, a, C3) for a in ALPHAS3}

    def step(k):
        a = ALPHAS3[k % len(ALPHAS3)]
        r = R.solve(Ab, p.b, *lams[a])
        return 1 if (r.converged and r.kkt1 <= TOL and r.kkt3 <= TOL) else 0

    for k in range(args.warmup):
        step(k)
    fits, t0 = 0, time.perf_counter()
    for k in range(args.steps):
        fits += step(k)
    dt = time.perf_counter() - t0
    value = fits / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("mixed form", "FP64 oracle on the stored BF16 values"),
                       "fits_per_step": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} oracle fits (alpha alternating 0.5, 0.9) of the workload, "
                                       f"NumPy/SciPy FP64 with {cores} BLAS threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _time_fits(pkg, ctx, b, steps, grid_per_alpha, stream):
    """Times `steps` steps of one fit per alpha on ctx with CUDA events on `stream`;
    returns (ms, fits, newton steps, last x per alpha (device), last results)."""
    import torch
    X = {a: torch.zeros((1, ctx.n), dtype=torch.float64, device="cuda") for a in grid_per_alpha}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fits = newton = 0
    last = {}
    for _ in range(steps):
        for a, grid in grid_per_alpha.items():
            st, res, done = pkg.ssnal_en_path(ctx.ctx, b, a, grid, X[a])
            fits += _count_fits(res, done)
            newton += sum(r.newton_iters for r in res[:done])
            last[a] = res[0]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), fits, newton, X, last


def _roofline(kernel, bytes_per_launch, ms, launches, peak, peak_kind, traffic=None, note=None):
    achieved = bytes_per_launch * launches / (ms / 1e3) / 1e9 if (ms > 0 and launches) else None
    out = {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": (achieved / peak) if achieved else None, "traffic": traffic, "traffic_unit": "bytes per launch",
           "peak_kind": peak_kind, "bytes_per_launch": bytes_per_launch, "timed_launches": launches,
           "avg_launch_us": (ms / launches * 1e3) if launches else None}
    if note:
        out["note"] = note
    return out


def run_path_headline(args, pkg, rank, world, local, barrier):
    """--workload path: the FP64 regularization path as the headline line (20 warm-started fits
    per step), with its e2e number through the C ABI (b in, all 20 solutions out)."""
    import torch
    from paper_2006_03970_gb300 import synth
    p = synth.config2(seed=SEED2, m=M2, n=N2)
    grid = list(synth.path_grid(K2, 0.05))
    ctx = pkg.Context(p.At)
    b = torch.as_tensor(p.b, dtype=torch.float64, device="cuda")
    X = torch.zeros((len(grid), ctx.n), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        pkg.ssnal_en_path(ctx.ctx, b, ALPHA2, grid, X)
    torch.cuda.synchronize()
    barrier()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    prof0 = pkg.ssnal_en_profile(ctx.ctx, True, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fits = newton = 0
    for _ in range(args.steps):
        st, res, done = pkg.ssnal_en_path(ctx.ctx, b, ALPHA2, grid, X)
        fits += _count_fits(res, done)
        newton += sum(r.newton_iters for r in res[:done])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    prof1 = pkg.ssnal_en_profile(ctx.ctx, False, False)
    clk = clocks.stop()
    ms, fits_all = reduce_over_ranks(e0.elapsed_time(e1), fits, "cuda")
    b_host = torch.empty(M2, dtype=torch.float64, pin_memory=True)
    b_host.copy_(torch.from_numpy(p.b))
    X_host = torch.empty((len(grid), ctx.n), dtype=torch.float64, pin_memory=True)
    bh, xh = b_host.numpy(), X_host.numpy()
    pkg.ssnal_en_path_host(ctx.ctx, bh, ALPHA2, grid, xh)
    barrier()
    t0 = time.perf_counter()
    efits = 0
    for _ in range(args.steps):
        st, res, done = pkg.ssnal_en_path_host(ctx.ctx, bh, ALPHA2, grid, xh)
        efits += _count_fits(res, done)
    edt, efits = reduce_over_ranks(time.perf_counter() - t0, efits, "cuda")
    peak, peak_kind = _peaks()
    rl = _roofline("k_stream_lane<kModeT, float pair> (t = A^T d over the pre-split copy, fused line-search trial "
                   "sums)", 8.0 * M2 * N2 + 3 * 8.0 * N2 + 8.0 * M2, prof1["stream_ms"], prof1["stream_launches"], peak,
                   peak_kind, TRAFFIC["split_modeT_m500_n1e5"])
    ctx.close()
    line = {"metric": "EN fits/s to KKT<=1e-6", "value": fits_all / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD2, "l2": "inputs larger than L2 (A is 400 MB, L2 129 MB)",
                       "fits_per_step": K2, "parallelism": "replicas" if world > 1 else "single GPU"},
            "clocks": clk, "e2e": {"value": efits / edt, "unit": UNIT, "h2d_bytes_per_step": 8 * M2,
                                   "d2h_bytes_per_step": 8 * len(grid) * N2},
            "gpu_launches": prof1["kernel_launches"] - prof0["kernel_launches"], "roofline": rl}
    if rank == 0:
        print(json.dumps(line))
    return 0


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

    if args.workload == "path":
        rc = run_path_headline(args, pkg, rank, world, local, barrier)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return rc
    p, bits = precision_problem()
    m, n = M3, N3
    ctx = pkg.Context(bits, dtype=pkg.BF16, options=pkg.ssnal_en_default_options(precision=1))
    b = torch.as_tensor(p.b, dtype=torch.float64, device="cuda")
    grids = {a: [C3] for a in ALPHAS3}
    stream = torch.cuda.current_stream()
    _time_fits(pkg, ctx, b, args.warmup, grids, stream)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)  # let the sampler start before the timed region
    prof0 = pkg.ssnal_en_profile(ctx.ctx, True, True)
    ms, fits, newton, Xm, last_m = _time_fits(pkg, ctx, b, args.steps, grids, stream)
    barrier()
    prof1 = pkg.ssnal_en_profile(ctx.ctx, False, False)
    phases = pkg.ssnal_en_profile_phases(ctx.ctx)
    clk = clocks.stop()
    ms, fits_all = reduce_over_ranks(ms, fits, "cuda")
    value = fits_all / (ms / 1e3)
    x_mixed = {a: Xm[a][0].cpu().numpy() for a in ALPHAS3}

    # end to end through the public C ABI with host buffers (b in, the solution out, per fit)
    b_host = torch.empty(m, dtype=torch.float64, pin_memory=True)
    b_host.copy_(torch.from_numpy(p.b))
    X_host = torch.empty((1, n), dtype=torch.float64, pin_memory=True)
    bh, xh = b_host.numpy(), X_host.numpy()
    for a in ALPHAS3:
        pkg.ssnal_en_path_host(ctx.ctx, bh, a, grids[a], xh)
    barrier()
    t0 = time.perf_counter()
    efits = 0
    for _ in range(args.steps):
        for a in ALPHAS3:
            st, res, done = pkg.ssnal_en_path_host(ctx.ctx, bh, a, grids[a], xh)
            efits += _count_fits(res, done)
    edt = time.perf_counter() - t0
    barrier()
    edt, efits = reduce_over_ranks(edt, efits, "cuda")
    e2e_value = efits / edt

    peak, peak_kind = _peaks()
    s_ms, s_n = prof1["stream_ms"], prof1["stream_launches"]
    u_ms, u_n = phases["u_refresh"]
    roofline = _roofline("k_stream_lane<kModeT, BF16> (t = A^T d over the stored BF16 values, FP32 accumulation, "
                         "fused line-search trial sums)", 2.0 * m * n + 3 * 8.0 * n + 8.0 * m, s_ms, s_n, peak,
                         peak_kind, TRAFFIC.get("bf16_modeT_m1000_n1e6"))
    roofline["launches"] = newton
    roofline["timed_every"] = 8
    roofline["share_of_step"] = (s_ms / s_n * newton / ms) if (ms > 0 and s_n) else None
    roofline_u = _roofline("k_stream_lane<kModeU, BF16 float-float> (u = A^T y over the stored BF16 values, "
                           "float-float accumulation)", 2.0 * m * n + 8.0 * n + 8.0 * m, u_ms, u_n, peak, peak_kind,
                           TRAFFIC.get("bf16ff_modeU_m1000_n1e6"))
    roofline_u["share_of_step"] = u_ms / ms if ms > 0 else None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "context": "paper Table S2 (m=1e3, n=1e6, alpha 0.9): 2.025 s per FP64 fit on a 2-core laptop CPU "
                       "(0.49 fits/s); another machine and generator, not the target",
            "precision": {"A": "BF16 storage", "newton_pass": "BF16 x FP32(d) products, FP32 accumulation",
                          "u_pass": "float-float (about 2^-46 relative)", "syrk": "BF16 tensor cores, FP32 accumulation",
                          "factor": "FP32 Cholesky + FP64 iterative refinement through the FP64 panel; FP64 "
                                    "Cholesky when the FP32 solve does not contract",
                          "kkt_gap_prox": "FP64"},
            "config": {"workload": WORKLOAD, "l2": "inputs larger than L2 (A is 2 GB BF16, L2 129 MB)",
                       "fits_per_step": len(ALPHAS3), "parallelism": "replicas" if world > 1 else "single GPU"},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * m * len(ALPHAS3),
                    "d2h_bytes_per_step": 8 * n * len(ALPHAS3)},
            "gpu_launches": prof1["kernel_launches"] - prof0["kernel_launches"],
            "roofline": roofline, "roofline_u_pass": roofline_u,
            "fits": {a: {"al_iters": r.al_iters, "newton_iters": r.newton_iters, "newton_fp64": r.newton_fp64,
                         "active": r.active, "kkt1": r.kkt1, "kkt3": r.kkt3} for a, r in last_m.items()}}
    ctx.close()
    del bits
    if rank == 0 and world == 1 and not args.no_fp64_form:
        line["fp64_form"], x_fp64 = fp64_form(pkg, p, grids, args.steps, args.warmup, stream, peak, peak_kind)
        line["mixed_over_fp64"] = value / line["fp64_form"]["value"] if line["fp64_form"]["value"] else None
    else:
        x_fp64 = None
    if rank == 0 and world == 1 and not args.no_oracle:
        line["oracle_errors"], line["cpu_baseline"] = oracle_errors(p, x_mixed, x_fp64)
    if rank == 0 and world == 1 and not args.no_path:
        line["fp64_path"] = path_workload(pkg, args.steps, args.warmup, peak, peak_kind)
    if rank == 0 and world == 1 and not args.no_batch:
        torch.cuda.empty_cache()  # give the library the memory the workloads above left cached
        line["batched"] = batched_fits()
        line["single_fit"] = small_fit()
    if rank == 0 and world == 1 and not args.no_serve:
        torch.cuda.empty_cache()
        line["serving"] = serve_workload(args.serve_requests, args.serve_matrices)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def fp64_form(pkg, p, grids, steps, warmup, stream, peak, peak_kind):
    """The headline workload with A stored as FP64 (the FP32 values, 8 GB) and solved in the
    FP64 form: float-float passes over the pre-split copy, FP32 factor + FP64 refinement."""
    import numpy as np
    import torch
    ctx = pkg.Context(np.asarray(p.At, dtype=np.float64))
    b = torch.as_tensor(p.b, dtype=torch.float64, device="cuda")
    _time_fits(pkg, ctx, b, warmup, grids, stream)
    pkg.ssnal_en_profile(ctx.ctx, True, True)
    ms, fits, newton, X, last = _time_fits(pkg, ctx, b, steps, grids, stream)
    prof = pkg.ssnal_en_profile(ctx.ctx, False, False)
    ctx.close()
    m, n = p.At.shape[1], p.At.shape[0]
    out = {"workload": "the headline workload with A stored as FP64 (8 GB; the FP32 values)", "value": fits / (ms / 1e3),
           "unit": UNIT, "ms_per_fit": ms / max(1, steps * len(grids)), "converged_fits": fits,
           "roofline": _roofline("k_stream_lane<kModeT, float pair> (t = A^T d, float-float over the pre-split copy)",
                                 8.0 * m * n + 3 * 8.0 * n + 8.0 * m, prof["stream_ms"], prof["stream_launches"], peak,
                                 peak_kind),
           "fits": {a: {"al_iters": r.al_iters, "newton_iters": r.newton_iters, "active": r.active, "kkt1": r.kkt1,
                        "kkt3": r.kkt3} for a, r in last.items()}}
    return out, {a: X[a][0].cpu().numpy() for a in X}


def _compare(At, b, lam1, lam2, x, ro):
    """Error of x against the oracle's solution ro.x on the problem (At, b, lam1, lam2)."""
    import numpy as np
    from oracle import checkers as C
    P_or = C.primal_objective(At, b, ro.x, lam1, lam2)
    P_x = C.primal_objective(At, b, x, lam1, lam2)
    xmax = np.abs(ro.x).max()
    big = np.abs(ro.x) > 1e-8 * max(xmax, 1e-300)
    return {"x_rel_inf": float(np.abs(x - ro.x).max() / max(xmax, 1e-300)),
            "obj_rel_gap": float(abs(P_x - P_or) / max(1.0, abs(P_or))),
            "support": [int(np.count_nonzero(x)), int(np.count_nonzero(ro.x))],
            "support_mismatch_outside_margin": int(np.count_nonzero(big & (x == 0)))}


def oracle_errors(p, x_mixed, x_fp64):
    """Errors against the FP64 oracle (outside the timed region): (i) the mixed form against
    the oracle on the stored BF16 values upcast to FP64 (solver error), (ii) the mixed form
    and the FP64 form against the oracle on the FP32 matrix (storage error and the FP64
    form's own parity).  The oracle fits on the stored values also give the CPU baseline."""
    import numpy as np
    from oracle import blas
    from oracle import ssnal_en_ref as R
    from paper_2006_03970_gb300 import synth
    cores = _cores()
    blas.set_blas_threads(cores)
    out = {"bars": {"obj_rel_gap": 1e-9, "x_rel_inf": 1e-6}, "stored_bf16": {}, "fp32_matrix": {}}
    Ab = _bf16_as_f64(synth.to_bf16_bits(p.At))
    t_or, fits = 0.0, 0
    for a in ALPHAS3:
        lam1, lam2 = R.lambdas(Ab, p.b, a, C3)
        t0 = time.perf_counter()
        ro = R.solve(Ab, p.b, lam1, lam2)
        t_or += time.perf_counter() - t0
        fits += 1 if (ro.converged and ro.kkt1 <= TOL and ro.kkt3 <= TOL) else 0
        out["stored_bf16"][str(a)] = {"mixed": _compare(Ab, p.b, lam1, lam2, x_mixed[a], ro),
                                      "oracle_al_iters": ro.al_iters, "oracle_newton_iters": ro.newton_iters}
    del Ab
    Af = np.ascontiguousarray(p.At, dtype=np.float64)
    for a in ALPHAS3:
        lam1, lam2 = R.lambdas(Af, p.b, a, C3)
        ro = R.solve(Af, p.b, lam1, lam2)
        e = {"mixed": _compare(Af, p.b, lam1, lam2, x_mixed[a], ro)}
        if x_fp64 is not None:
            e["fp64_form"] = _compare(Af, p.b, lam1, lam2, x_fp64[a], ro)
        out["fp32_matrix"][str(a)] = e
    cpu = {"value": fits / t_or, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"one oracle fit per alpha (0.5, 0.9) of the headline workload on the stored BF16 values "
                     f"upcast to FP64, NumPy/SciPy FP64 with {cores} BLAS threads", "seconds": t_or}
    return out, cpu


def path_workload(pkg, steps, warmup, peak, peak_kind):
    """The FP64 regularization path of the path configuration (20 warm-started fits per step)."""
    import torch
    from paper_2006_03970_gb300 import synth
    p = synth.config2(seed=SEED2, m=M2, n=N2)
    grid = list(synth.path_grid(K2, 0.05))
    ctx = pkg.Context(p.At)
    b = torch.as_tensor(p.b, dtype=torch.float64, device="cuda")
    X = torch.zeros((len(grid), ctx.n), dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        pkg.ssnal_en_path(ctx.ctx, b, ALPHA2, grid, X)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    pkg.ssnal_en_profile(ctx.ctx, True, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fits = newton = 0
    for _ in range(steps):
        st, res, done = pkg.ssnal_en_path(ctx.ctx, b, ALPHA2, grid, X)
        fits += _count_fits(res, done)
        newton += sum(r.newton_iters for r in res[:done])
    e1.record(stream)
    torch.cuda.synchronize()
    prof = pkg.ssnal_en_profile(ctx.ctx, False, False)
    ctx.close()
    ms = e0.elapsed_time(e1)
    rl = _roofline("k_stream_lane<kModeT, float pair> (t = A^T d over the pre-split copy, fused line-search trial "
                   "sums)", 8.0 * M2 * N2 + 3 * 8.0 * N2 + 8.0 * M2, prof["stream_ms"], prof["stream_launches"], peak,
                   peak_kind, TRAFFIC["split_modeT_m500_n1e5"])
    rl["share_of_step"] = (prof["stream_ms"] / prof["stream_launches"] * newton / ms) if prof["stream_launches"] else None
    return {"workload": WORKLOAD2, "value": fits / (ms / 1e3), "unit": UNIT, "ms_per_path": ms / steps,
            "converged_fits": fits, "newton_steps": newton, "roofline": rl}


def batched_fits(count=512):
    """The batched configuration: 512 independent fits, m log-uniform in [50, 500], n log-uniform in
    [1e3, 5e4], A iid N(0,1) standardized and stored in FP32, max(5, m/20) nonzeros, snr 5,
    alpha 0.7, c ~ U[0.2, 0.8] (seed 4).  All matrices are resident; each timed batch starts from
    x = 0.  Reported: fits/s of ssnal_en_solve_batch_resident (one persistent kernel: each CTA
    runs whole fits from a device work queue, largest first, with the loads in flight of its
    passes over A tuned on the batch), of ssnal_en_solve_batch (host worker threads with their
    own streams, tuned worker count) and of the same instances solved one after another."""
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
    fits = [(c.A, c.m, b, l1, l2, x) for c, b, (l1, l2), x in zip(ctxs, bs, lams, xs)]

    def reset():
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()

    def ok_count(res):
        return sum(1 for r in res if r.status == 0 and r.kkt1 <= TOL and r.kkt3 <= TOL)

    reset()
    pkg.ssnal_en_solve_batch_resident(fits)  # warm-up
    reset()
    t0 = time.perf_counter()
    st, res_d, info = pkg.ssnal_en_solve_batch_resident(fits)
    dt_d = time.perf_counter() - t0
    ok_d = ok_count(res_d)
    x_dev = [x.clone() for x in xs]
    reset()
    pkg.ssnal_en_solve_batch(inst, 0)  # warm-up (and tuning)
    reset()
    t0 = time.perf_counter()
    st, res, used = pkg.ssnal_en_solve_batch(inst, 0)
    dt = time.perf_counter() - t0
    ok = ok_count(res)
    # the two batch paths take different kernels: agreement of the solutions (relative)
    agree = max(float((a - b).abs().max()) / max(float(b.abs().max()), 1e-300) for a, b in zip(x_dev, xs))
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
            "fits_per_s": ok_d / dt_d, "seconds": dt_d, "converged": ok_d,
            "resident": {"kernel": "k_batch_solve (persistent, one CTA per SM, device work queue)",
                         "loads_in_flight": info[0], "fits_on_regular_path": info[1]},
            "threaded_fits_per_s": ok / dt, "threaded_seconds": dt, "threaded_converged": ok, "workers": used,
            "max_rel_diff_resident_vs_threaded": agree, "sequential_fits_per_s": count / dts}


def small_fit(reps=200, copies=None):
    """The single-fit configuration: m=100, n=2000, iid N(0,1) standardized, 10 nonzeros
    +-U[1,3], snr 5, alpha 0.8, c 0.5, seed 0, FP64 -- a fit bound by launch latency.
    Reported: ms per fit of ssnal_en_solve (FP64 storage, each fit from x = 0, one after
    another), and of the device-resident solver (ssnal_en_solve_batch_resident) on the same
    matrix stored in FP32: one fit per launch (latency) and one copy per SM in one launch
    (throughput of independent fits of this size)."""
    import numpy as np
    import torch
    import paper_2006_03970_gb300 as pkg
    from paper_2006_03970_gb300 import synth
    p = synth.config1()
    m, n = p.At.shape[1], p.At.shape[0]
    g = np.abs(p.At @ p.b).max()
    l1, l2 = p.c * g, (1 - p.alpha) / p.alpha * p.c * g
    ctx = pkg.Context(p.At)
    b = torch.as_tensor(p.b, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    for _ in range(5):
        x.zero_()
        pkg.ssnal_en_solve(ctx.ctx, b, l1, l2, x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    kkt = 0.0
    for _ in range(reps):
        x.zero_()
        st, r = pkg.ssnal_en_solve(ctx.ctx, b, l1, l2, x)
        kkt = max(kkt, r.kkt1, r.kkt3)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    x_reg = x.clone()
    ctx.close()
    A32 = torch.as_tensor(np.ascontiguousarray(p.At, dtype=np.float32), device="cuda")
    copies = copies or torch.cuda.get_device_properties(0).multi_processor_count
    xs = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(copies)]
    one = [(A32, m, b, l1, l2, xs[0])]
    for _ in range(5):
        xs[0].zero_()
        pkg.ssnal_en_solve_batch_resident(one)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        xs[0].zero_()
        st, res1, info1 = pkg.ssnal_en_solve_batch_resident(one)
    torch.cuda.synchronize()
    dt1 = (time.perf_counter() - t0) / reps
    many = [(A32, m, b, l1, l2, xx) for xx in xs]
    for xx in xs:
        xx.zero_()
    pkg.ssnal_en_solve_batch_resident(many)
    for xx in xs:
        xx.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, resm, infom = pkg.ssnal_en_solve_batch_resident(many)
    torch.cuda.synchronize()
    dtm = time.perf_counter() - t0
    okm = sum(1 for r in resm if r.status == 0 and r.kkt1 <= TOL and r.kkt3 <= TOL)
    diff = float((xs[0] - x_reg).abs().max()) / max(float(x_reg.abs().max()), 1e-300)
    return {"workload": "m=100, n=2000, iid N(0,1) standardized, 10 nonzeros +-U[1,3], snr 5, alpha 0.8, c 0.5, "
                        "tol 1e-6, seed 0",
            "fits_per_s": 1.0 / dt, "ms_per_fit": 1e3 * dt, "storage": "FP64", "max_kkt": kkt,
            "resident_one_fit": {"ms_per_fit": 1e3 * dt1, "fits_per_s": 1.0 / dt1, "storage": "FP32",
                                 "active": res1[0].active, "newton_iters": res1[0].newton_iters},
            "resident_copies": {"copies": copies, "seconds": dtm, "fits_per_s": okm / dtm, "converged": okm},
            "max_rel_diff_resident_fp32_vs_fp64": diff}


def serve_workload(per_rate=400, n_small=16, workers=16, seed=5, keep=None, group=8):
    """The serving configuration: a resident genotype-like A (m=2000, n=500000 codes
    ~ Binomial(2, p_j), p_j ~ U(0.05, 0.5), stored four per byte, standardized on the fly by
    per-column FP32 mean and scale) plus `n_small` resident FP32 matrices from the precision workload's generator (m
    log-uniform in [200, 1000], n log-uniform in [1e4, 2e5], 50-feature blocks rho 0.5).  Each
    request: its own x* (30 nonzeros +-U[0.5, 2]), b = A x* + noise at snr 2, alpha ~ U[0.5, 1),
    c ~ U[0.1, 0.8]; its matrix is the genotype one with probability 1/2, else uniform over the
    others.  The server runs the mixed form (precision 1) with `workers` worker streams, each
    advancing up to `group` requests on one matrix together with their passes over A merged
    (A^T [d_1 ... d_k]); requests arriving on that matrix join as places free up.  First a
    burst of `per_rate` requests gives the saturation throughput; then Poisson arrivals at
    {0.25, 0.5, 0.75, 0.9, 1.1} x that rate, `per_rate` requests each, give latency percentiles
    (submission to completion, host transfers included).  Each phase also reports how many
    requests needed the FP64 Newton system (newton_fp64 > 0) and lists the unconverged ones;
    `keep` (a list) receives (matrix index, b, alpha, c, result) of those requests."""
    import math
    import numpy as np
    import torch
    import paper_2006_03970_gb300 as pkg
    from paper_2006_03970_gb300 import synth
    rng = np.random.Generator(np.random.PCG64(seed))
    codes, mean, scale = synth.genotype_matrix(2000, 500_000, seed=seed)
    Ag, mg = pkg.device_matrix(codes, pkg.I2_GENO)  # four codes per byte: 250 MB per pass
    mats = [(Ag, mg, pkg.I2_GENO, torch.as_tensor(mean, device="cuda"), torch.as_tensor(scale, device="cuda"))]
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

    srv = pkg.Server(mats, workers=workers, options=pkg.ssnal_en_default_options(precision=1), group=group)

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
        conv = [g[1].status == 0 and g[1].kkt1 <= TOL and g[1].kkt3 <= TOL for g in got]
        unconverged = []
        for (k, b, alpha, c), g, ok_i in zip(reqs, got, conv):
            if not ok_i:
                unconverged.append({"matrix": k, "m": sizes[k][0], "n": sizes[k][1], "alpha": alpha, "c": c,
                                    "status": g[1].status, "kkt1": g[1].kkt1, "kkt3": g[1].kkt3,
                                    "al_iters": g[1].al_iters, "newton_iters": g[1].newton_iters})
            if keep is not None and (not ok_i or g[1].newton_fp64 > 0):
                keep.append((k, b, alpha, c, g[1].as_dict()))
        return {"requests": len(reqs), "converged": sum(conv), "fits_per_s": sum(conv) / span,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "fp64_newton_requests": sum(1 for g in got if g[1].newton_fp64 > 0), "unconverged": unconverged}

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
    if keep is not None:
        keep.append(("matrices", mats, host_cols, sizes))
    return {"workload": f"resident genotype A 2000x500000 2-bit codes (250 MB) + {n_small} FP32 matrices "
                        f"(m in [200,1000], n in [1e4,2e5]); requests 50% genotype, alpha ~ U[0.5,1), "
                        f"c ~ U[0.1,0.8], x* 30 nonzeros, snr 2; mixed form, {workers} worker streams, groups of "
                        f"up to {group} requests per matrix with merged passes over A",
            "saturation": burst, "poisson_sweep": sweep}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["precision", "path"], default="precision",
                    help="headline workload: the precision configuration (default) or the FP64 path "
                         "(path: the headline line only)")
    ap.add_argument("--no-oracle", "--no-cpu-baseline", action="store_true",
                    help="skip the oracle errors and the CPU baseline")
    ap.add_argument("--no-fp64-form", "--no-mixed", action="store_true",
                    help="skip the FP64 form of the headline workload")
    ap.add_argument("--no-path", action="store_true", help="skip the FP64 regularization path workload")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--serve-requests", type=int, default=1667,
                    help="requests per serving phase (burst + 5 arrival rates: 10,002 in all)")
    ap.add_argument("--serve-matrices", type=int, default=64, help="resident FP32 matrices (serving)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
