"""Benchmark: exact GP log-likelihood evaluations per second on one GB300 (and N independent replicas).

One step = one full evaluation of the hot path for a new hyperparameter setting on a cached point set:
A3 bump features, A4 kernel values into the supernodal panels, A7 numeric factorization, A8-A10 solves,
log-determinant and log-likelihood (A11 refinement in mixed precision). The point-set steps A1, A2, A5, A6
(cell list, pattern, ordering, symbolic analysis) are cached per point set and run before timing.

Default workload: station space-time field, 5000 sites from a seeded 50-component Gaussian mixture on [0,1]^2
times 240 daily steps (n = 1.2M), 16 bumps (4 x 4, spatial), Wendland core with radii set for ~100 nonzeros per
row, noise variance 0.25. Inputs are synthetic and seeded; factor and workspace are tens of GB, far larger
than the 126 MB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--precision mixed|fp64]
       python bench.py --impl reference ...    (the CPU oracle, timed on a bounded sample of the workload)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP64 FMA throughput of a GB300 of this machine, measured with a dependent-free FP64 FMA loop over all SMs (the FP64
# path's A7 kernels are bound by it; FP64 tensor-core DMMA measured no faster on this part)
MEASURED_FP64_TFLOPS = 1.011
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def make_workload(name: str):
    from paper_2411_05869_gb300 import synth
    if name == "station_1.2M":   # with the 200 x 200 x 30 prediction grid
        return synth.config(5, with_test=True)
    if name == "station_120k":   # the same field over the first 24 days: a profiling-size case
        return synth.station_spacetime(nsites=5000, ndays=24, with_test=False)
    if name == "spacetime_100k":
        return synth.config(2, m=0)
    if name == "batched_200k":
        return synth.uniform_spacetime(200_000, 0, 80.0, 8, seed=synth.SEED_BASE + 3, name="spacetime_200k")
    if name == "noncompact_50k":   # the non-compact core of App. B on 2-D points (pattern: the support of C_sparse)
        return synth.noncompact_spatial(50_000, seed=synth.SEED_BASE + 6)
    if name == "spatial_2k":   # the residual is the workload's seeded normals (its GP draw is left to the caller)
        w = synth.spatial_2d(n=2000, m=0, seed=synth.SEED_BASE + 1)
        w.resid = w.normals.copy()
        return w
    raise SystemExit(f"unknown workload {name}")


def workload_config(w, name, precision, extra=None):
    hp = w.hyper
    cfg = {"workload": name, "n": int(w.X.shape[0]), "d": int(hp.d), "bumps": f"{hp.n1}x{hp.n2}",
           "bump_dims": int(hp.bump_dims), "core_radius": [float(x) for x in hp.core_radius],
           "noise_var": float(hp.noise_var), "precision": precision, "B": 1,
           "l2": "inputs larger than L2 (factor and workspace >> 126 MB), no flush"}
    if extra:
        cfg.update(extra)
    return cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------ oracle leg

def oracle_sample(w, max_points: int = 30_000):
    """A bounded sub-window of the workload for the CPU oracle. Station workloads keep every site (the spatial
    density and hence the neighbour counts of the full field) over the first few days; other workloads take
    the first points in index order (the same law)."""
    n = w.X.shape[0]
    if n <= max_points:
        return w.X, w.resid, "whole workload"
    if "nsites" in w.info:
        ns, nd = w.info["nsites"], w.info["ndays"]
        days = max(1, min(nd, max_points // ns))
        idx = (np.arange(ns)[:, None] * nd + np.arange(days)[None, :]).ravel()
        return w.X[idx], w.resid[idx], f"all {ns} sites x the first {days} days ({idx.size} points) of the field"
    idx = np.arange(max_points)
    return w.X[idx], w.resid[idx], f"first {max_points} of {n} points (same law)"


class OracleLeg:
    """The CPU oracle on a bounded sample: pattern, ordering and symbolic analysis once (cached, like the GPU
    path's point set), then one sparse log-likelihood per step for a new hyperparameter setting. Rates are
    projected to the full workload by the flop ratio sum_j eta_j^2 (full) / sum_j eta_j^2 (sample)."""

    def __init__(self, w, max_points: int, full_flops: float):
        import oracle
        self.oracle = oracle
        self.X, self.r, self.desc = oracle_sample(w, max_points)
        self.hp = w.hyper
        t0 = time.perf_counter()
        if int(getattr(self.hp, "core_kind", 0)) == 1:   # non-compact core: the support of C_sparse
            self.rp, self.col = oracle.pattern_sparse(self.hp, self.X)
            self.perm = oracle.fill_order(self.X, self.hp.r0, self.rp, self.col)
        else:
            self.rp, self.col = oracle.pattern(self.X, self.hp.core_radius)
            self.perm = oracle.fill_order(self.X, self.hp.core_radius, self.rp, self.col)
        sym = oracle.symbolic(self.rp, self.col, self.perm, want_rows=False)
        self.t_setup = time.perf_counter() - t0
        self.sample_flops = float((sym["eta"].astype(np.float64) ** 2).sum())
        self.scale = max(full_flops / self.sample_flops, 1.0) if full_flops > 0 else 1.0

    def step(self, theta) -> float:
        t0 = time.perf_counter()
        self.last = self.oracle.sparse_loglik(theta, self.X, self.rp, self.col, self.perm, self.r)["loglik"]
        return time.perf_counter() - t0

    def step_threads(self, thetas, threads: int) -> float:
        """One evaluation per setting, `threads` at a time on host threads (the oracle's C call releases the
        interpreter lock, so the evaluations run in parallel); returns the wall time of all of them."""
        import concurrent.futures as cf
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda th: self.oracle.sparse_loglik(th, self.X, self.rp, self.col, self.perm, self.r),
                        thetas))
        return time.perf_counter() - t0

    def describe(self, t_eval: float) -> str:
        return (f"{self.desc}; oracle sparse loglik {t_eval:.2f} s per evaluation ({self.sample_flops:.3g} flops), "
                f"projected to the full workload by the flop ratio x{self.scale:.4g}")


def host_cpu():
    """The host's cores and CPU model (the oracle baseline runs there)."""
    model = None
    try:
        for ln in open("/proc/cpuinfo"):
            key = ln.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model or "unknown"}


def subwindow_parity(ctx, leg, theta, prec_list):
    """The GPU path on the oracle leg's sub-window, against the oracle's log-likelihood for the same setting."""
    import torch
    from paper_2411_05869_gb300 import gp
    dev = torch.device("cuda", ctx.device)
    st = ctx.stream
    with torch.cuda.stream(st):
        X = torch.as_tensor(leg.X, dtype=torch.float64, device=dev)
        r = torch.as_tensor(leg.r, dtype=torch.float64, device=dev)
    st.synchronize()
    if int(getattr(theta, "core_kind", 0)) == 1:
        ps = ctx.assemble_sparse_support(X, theta)
    else:
        ps = ctx.assemble(X, theta.core_radius)
    ref = leg.oracle.sparse_loglik(theta, leg.X, leg.rp, leg.col, leg.perm, leg.r)["loglik"]
    out = {"points": int(leg.X.shape[0]), "oracle_loglik": float(ref),
           "structure_bit_exact": bool(np.array_equal(ps.export("col"), leg.col) and
                                       np.array_equal(ps.export("perm"), leg.perm))}
    for name, prec in prec_list:
        f = ctx.factor(ps, [theta], prec)
        with torch.cuda.stream(st):
            o = f.loglik(r)
        st.synchronize()   # the log-likelihood is written on the library's stream
        ll = float(o.cpu()[0])
        f.free()
        out[f"{name}_loglik"] = ll
        out[f"{name}_rel_err"] = abs(ll - ref) / abs(ref)
    ps.free()
    return out


# ------------------------------------------------------------------------------------------------ GPU leg

def max_over_ranks(x: float, device) -> float:
    """The largest of every rank's x (all ranks call it; torch.distributed is initialised)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Units all ranks processed (each rank the same number: weak scaling) per second of the slowest rank."""
    return units_per_rank * world / max_seconds


def other_split_leg(ctx, ps, stream, resid, thetas, args, steps=3, warmup=2):
    """One setting per step through a factor with the other operand split (GP_OPT_SPLIT_F16 flipped)."""
    import torch
    from paper_2411_05869_gb300 import gp
    split = 1 - int(args.split_f16)
    ctx.set_option("split_f16", split)
    try:
        f2 = ctx.factor(ps, thetas[:1], gp.GP_MIXED)
    finally:
        ctx.set_option("split_f16", int(args.split_f16))
    out = torch.empty(1, dtype=torch.float64, device=resid.device)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    with torch.cuda.stream(stream):
        for k in range(warmup):
            f2.update([thetas[(1 + k) % len(thetas)]])
            f2.loglik(resid, out=out)
        evs[0].record(stream)
        for k in range(steps):
            f2.update([thetas[(1 + warmup + k) % len(thetas)]])
            f2.loglik(resid, out=out)
            evs[k + 1].record(stream)
        f2.update(thetas[:1])
        f2.loglik(resid, out=out)
    stream.synchronize()
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    ll = float(out.cpu()[0])
    f2.free()
    return {"operand_split": "fp16 pairs" if split else "tf32 pairs", "evals_per_s": 1e3 / float(np.mean(per)),
            "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99)),
                           "steps": steps},
            "loglik": ll, "note": "the same point set, blocking and settings with the other operand split of the "
                                  "tensor-core updates; loglik is that of the FP64 comparison's setting"}


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2411_05869_gb300 import gp

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = make_workload(args.workload)
    hp = w.hyper
    prec = gp.GP_MIXED if args.precision == "mixed" else gp.GP_FP64
    stream = torch.cuda.Stream(device=dev)
    ctx = gp.Context(local_rank, stream=stream)
    ctx.set_option("diag_fp32", int(args.diag_fp32))
    ctx.set_option("split_f16", int(args.split_f16))
    with torch.cuda.stream(stream):
        X = torch.as_tensor(w.X, dtype=torch.float64, device=dev)
        resid = torch.as_tensor(w.resid, dtype=torch.float64, device=dev)
    stream.synchronize()
    t0 = time.perf_counter()
    if int(getattr(hp, "core_kind", 0)) == 1:
        ps = ctx.assemble_sparse_support(X, hp)
    else:
        ps = ctx.assemble(X, hp.core_radius)
    t_assemble = time.perf_counter() - t0
    info = ps.info()
    rng = np.random.default_rng(1234 + rank)
    from paper_2411_05869_gb300 import synth
    B = max(1, args.batch)
    # proposals per factorization: all B when they fit, else B split evenly over the fewest factorizations whose
    # chunks fit in 80 % of free memory (every step evaluates exactly B settings when Bc divides B)
    per = ps.factor_bytes(hp, 1, prec)
    free = torch.cuda.mem_get_info(dev)[0]
    Bmax = max(1, min(B, int(0.8 * free) // per))
    nchunk = (B + Bmax - 1) // Bmax
    Bc = (B + nchunk - 1) // nchunk
    thetas = [synth.perturb(rng, hp, 0.05 if B == 1 else 0.1) for _ in range(B * (args.steps + args.warmup + 2))]
    tune = None
    if prec == gp.GP_MIXED and args.blocking:   # a fixed update blocking (group blocks, group tile width)
        g, tn = (int(v) for v in args.blocking.split(","))
        ps.set_blocking(g, tn)
        tune = {"chosen": {"group_blocks": g, "group_tile_n": tn}, "fixed": True}
    elif prec == gp.GP_MIXED and args.autotune:   # update blocking chosen by timing factorizations of Bc settings
        t0 = time.perf_counter()
        tried = ps.autotune(thetas[:Bc], reps=1)
        best = min(tried, key=lambda t: t["ms"])
        tune = {"chosen": {"group_blocks": best["group_blocks"], "group_tile_n": best["group_tile_n"]},
                "candidates": tried, "seconds": round(time.perf_counter() - t0, 2)}
    f = ctx.factor(ps, thetas[:Bc], prec)
    out = torch.empty(Bc, dtype=torch.float64, device=dev)
    resid_b = resid.expand(Bc, -1).contiguous() if Bc > 1 else resid

    def step(i):   # one evaluation of each of the B proposals of step i
        for c in range(nchunk):
            k0 = (i * B + c * Bc) % len(thetas)
            f.update([thetas[(k0 + j) % len(thetas)] for j in range(Bc)])
            f.loglik(resid_b, out=out)

    # warm-up
    for i in range(args.warmup):
        step(i)
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    f.info()
    launches0 = ctx.launches()
    clocks = ClockSampler(local_rank)
    clocks.start()
    stream.synchronize()
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(args.steps):
            step(args.warmup + k)
            ev[k + 1].record(stream)
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    f.info()   # adds the refinement loop's device-decided passes to the launch count
    launches = ctx.launches() - launches0
    per_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[args.steps])
    ll_last = float(out.cpu()[0])

    # end to end through the public API from host buffers: H2D of r from pinned memory, theta structs from
    # the host, D2H of the log-likelihood, every step
    r_host = torch.from_numpy(np.tile(w.resid, (Bc, 1)).reshape(tuple(resid_b.shape))).pin_memory()
    out_host = torch.empty(Bc, dtype=torch.float64).pin_memory()
    r_dev = torch.empty_like(resid_b)
    e2e_steps = max(1, min(args.steps, 5))
    stream.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(e2e_steps):
            for c in range(nchunk):
                r_dev.copy_(r_host, non_blocking=True)
                f.update([thetas[(k * B + c * Bc + j) % len(thetas)] for j in range(Bc)])
                f.loglik(r_dev, out=out)
                out_host.copy_(out, non_blocking=True)
                stream.synchronize()
    e2e_s = time.perf_counter() - t0

    # A12 predictive mean on the workload's test points (the 200 x 200 x 30 grid at 1.2M) for the last setting,
    # timed separately from the log-likelihood steps
    if w.Xtest is not None and w.Xtest.shape[0] > 0:
        Xt = torch.as_tensor(w.Xtest, dtype=torch.float64, device=dev)
        mut = torch.as_tensor(w.mu_test, dtype=torch.float64, device=dev)
        mean = torch.empty(Xt.shape[0], dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            f.predict(Xt, mut, out=mean)   # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                f.predict(Xt, mut, out=mean)
            e1.record(stream)
        stream.synchronize()
        pms = e0.elapsed_time(e1) / 3
        predict_info = {"m": int(Xt.shape[0]), "ms": pms, "points_per_s": Xt.shape[0] / (pms * 1e-3),
                        "finite": bool(torch.isfinite(mean).all().item())}
    else:
        predict_info = None

    # predictive variance diag(C_{y|z}) on the first test points of the workload (the grid's first cells; the
    # whole grid would take the printed projection), timed like the mean
    var_info = None
    if w.Xtest is not None and w.Xtest.shape[0] > 0 and args.var_points > 0:
        mv = min(args.var_points, w.Xtest.shape[0])
        Xv = torch.as_tensor(w.Xtest[:mv], dtype=torch.float64, device=dev)
        var = torch.empty(mv, dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            f.predict_var(Xv[:min(mv, 256)], out=var[:min(mv, 256)])   # warm-up (allocates the workspace)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f.predict_var(Xv, out=var)
            e1.record(stream)
        stream.synchronize()
        vms = e0.elapsed_time(e1)
        vv = var.cpu().numpy()
        var_info = {"m": int(mv), "ms": vms, "points_per_s": mv / (vms * 1e-3),
                    "grid_projection_s": w.Xtest.shape[0] / (mv / (vms * 1e-3)),
                    "min": float(vv.min()), "max": float(vv.max()), "positive": bool((vv > 0).all()),
                    "note": "first test points of the workload's grid; FP32 solves with the mixed factor" if
                    prec == gp.GP_MIXED else "first test points of the workload's grid; FP64 factor"}

    # the paper's own iterative computation (stochastic Lanczos log-det, MINRES at 1e-8) on the same C_z values,
    # against this step's exact result for the same setting
    it_info = None
    if args.iterative_probes > 0:
        ths0 = thetas[:1]
        g = np.random.default_rng(77)
        pr = torch.as_tensor(g.choice([-1.0, 1.0], size=(args.iterative_probes, w.X.shape[0])), device=dev)
        x0 = torch.as_tensor(g.standard_normal(w.X.shape[0]), device=dev)
        with torch.cuda.stream(stream):
            f.update([ths0[0]] * Bc)
            exact = f.loglik(resid_b, out=out)
        stream.synchronize()
        ll_exact = float(out.cpu()[0])
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            itr = f.loglik_iterative(resid, pr, x0, lanczos_steps=args.iterative_steps, tol=1e-8)
        it_s = time.perf_counter() - t0
        it_info = {"probes": args.iterative_probes, "lanczos_steps": args.iterative_steps, "tol": 1e-8,
                   "seconds": it_s, "loglik": itr["loglik"], "exact_loglik": ll_exact,
                   "loglik_rel_diff": abs(itr["loglik"] - ll_exact) / abs(ll_exact), "logdet": itr["logdet"],
                   "minres_iters": itr["minres_iters"], "converged": bool(itr["converged"]),
                   "true_relres": itr["true_relres"],
                   "note": "the paper's approximate path (Sec. 3.3) on the factor's C_z values; the exact "
                           "log-likelihood is this run's mixed evaluation of the same setting"}

    # per-kernel-class profile of one more step (not part of the timed region)
    ctx.profile(True)
    step(0)
    stream.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)

    # settings of the batched leg, evaluated one at a time here for the comparison with their batched results
    leg_B = args.batch_leg if (prec == gp.GP_MIXED and B == 1 and args.batch_leg > 1) else 0
    leg_single = None
    if leg_B:
        per_leg = ps.factor_bytes(hp, leg_B, prec)
        while leg_B > 1 and per_leg > args.batch_leg_budget_gb * 1e9:
            leg_B -= 1
            per_leg = ps.factor_bytes(hp, leg_B, prec)
        leg_thetas = [synth.perturb(rng, hp, 0.05) for _ in range(leg_B * (args.batch_leg_steps + 1))]
        leg_single = []
        for th in leg_thetas[:leg_B]:
            with torch.cuda.stream(stream):
                f.update([th])
                f.loglik(resid, out=out)
            stream.synchronize()   # out is written on the library's stream
            leg_single.append(float(out.cpu()[0]))

    res = dict(total_ms=total_ms, per=per_ms, launches=launches, B=B, Bc=Bc, nchunk=nchunk, predict=predict_info,
               variance=var_info, iterative=it_info,
               autotune=tune, clk=clk, info=info, t_assemble=t_assemble,
               e2e_s=e2e_s, e2e_steps=e2e_steps, n=int(w.X.shape[0]), prof=prof, ll=ll_last,
               h2d=int(w.resid.nbytes) * Bc * nchunk, d2h=8 * Bc * nchunk, w=w)
    # the other operand split of the tensor-core updates (TF32 pairs beside FP16 pairs, or the reverse) on the same
    # point set and blocking: steady-state steps timed like the main ones, and the log-likelihood of the setting the
    # FP64 comparison takes
    if prec == gp.GP_MIXED and B == 1 and args.other_split:
        res["other_split"] = other_split_leg(ctx, ps, stream, resid, thetas, args)
    # FP64 comparison (mixed runs only): the same settings through the FP64 path. The factor is created (allocated
    # and factored once) outside the timing; then --fp64-steps steady-state steps of update + loglik are timed
    # with CUDA events, like the mixed steps, for p50/p99.
    if prec == gp.GP_MIXED and args.fp64_steps > 0:
        nb = min(Bc, args.fp64_proposals)
        ths = thetas[:Bc]
        f.update(ths)
        f.loglik(resid_b, out=out)
        stream.synchronize()   # out is written on the library's stream
        ll_mixed = out.cpu().numpy()[:nb].copy()
        f.free()   # room for the FP64 factor
        r64 = resid_b[:nb] if nb > 1 else resid
        stream.synchronize()
        with torch.cuda.stream(stream):
            f64 = ctx.factor(ps, ths[:nb], gp.GP_FP64)
            out64 = f64.loglik(r64)
            stream.synchronize()
            ll64 = out64.cpu().numpy()
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.fp64_steps + 1)]
            evs[0].record(stream)
            for k in range(args.fp64_steps):
                f64.update(ths[:nb])
                f64.loglik(r64, out=out64)
                evs[k + 1].record(stream)
        stream.synchronize()
        per64 = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.fp64_steps)]
        rel = np.abs(ll_mixed - ll64) / np.abs(ll64)
        if "other_split" in res:
            o = res["other_split"]
            o["mixed_rel_diff_vs_fp64"] = abs(o["loglik"] - float(ll64[0])) / abs(float(ll64[0]))
        res["fp64"] = {"ms_per_step": float(np.mean(per64)) / nb, "evals_per_s": nb * 1e3 / float(np.mean(per64)),
                       "latency_ms": {"p50": float(np.percentile(per64, 50)), "p99": float(np.percentile(per64, 99)),
                                      "steps": len(per64)},
                       "loglik": float(ll64[0]), "mixed_loglik": float(ll_mixed[0]),
                       "mixed_rel_diff": float(rel.max()), "proposals_compared": int(nb),
                       "mixed_rel_diff_per_proposal": [float(x) for x in rel] if nb > 1 else None,
                       "note": f"FP64 path on {nb} of the settings: steady-state update + loglik steps (factor "
                               "created before timing); mixed_rel_diff is the largest over the settings"}
        f64.free()
        f = None
    if f is not None:
        f.free()
    if leg_B > 1:   # leg_B settings in one factorization and one batched solve per step, within the budget
        res["batched"] = batched_leg(ctx, ps, stream, resid, leg_thetas, leg_single, leg_B, args.batch_leg_steps,
                                     per_leg, args.batch_leg_budget_gb)
    ps.free()
    res["ctx"] = ctx
    return res


def batched_leg(ctx, ps, stream, resid, thetas, single, Bl, steps, nbytes, budget_gb):
    """Bl settings per factorization on the same point set: every launch of A3-A11 spans all Bl. One warm-up
    step, then `steps` timed steps (new settings each step) with CUDA events; the first step's settings are also
    compared with their one-at-a-time evaluations."""
    import torch
    from paper_2411_05869_gb300 import gp
    dev = resid.device
    fb = ctx.factor(ps, thetas[:Bl], gp.GP_MIXED)
    rb = resid.expand(Bl, -1).contiguous()
    outb = torch.empty(Bl, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        fb.loglik(rb, out=outb)
    stream.synchronize()
    llb = outb.cpu().numpy().copy()
    rel = [abs(a - b) / abs(b) for a, b in zip(llb, single)]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(steps):
            fb.update(thetas[(k + 1) * Bl:(k + 2) * Bl])
            fb.loglik(rb, out=outb)
            ev[k + 1].record(stream)
    stream.synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    ctx.profile(True)
    fb.update(thetas[:Bl])
    fb.loglik(rb, out=outb)
    stream.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    fb.free()
    return {"B": Bl, "steps": steps, "evals_per_s": Bl * steps * 1e3 / sum(per), "ms_per_step": float(np.mean(per)),
            "ms_per_eval": float(np.mean(per)) / Bl,
            "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
            "factor_bytes": int(nbytes), "budget_gb": budget_gb,
            "rel_diff_vs_one_at_a_time": float(max(rel)),
            "kernels_ms": {k: round(v[0], 3) for k, v in prof.items()},
            "note": f"{Bl} settings per factorization (every launch spans all of them); steady-state update + loglik "
                    "steps timed with CUDA events; rel_diff compares the first step's log-likelihoods with the same "
                    "settings evaluated one at a time"}


# ------------------------------------------------------------------------------------------------ MCMC leg

def run_mcmc(args):
    """The App. C sampler on the 200k-point batched workload: `--batch` lockstep chains (default 16), every block
    update one batched factorization and solve of all chains (the mean block solves only). Times --steps full
    iterations after --warmup, with the mixed path and the autotuner's blocking."""
    import torch
    from paper_2411_05869_gb300 import gp, mcmc
    w = make_workload("batched_200k")
    hp = w.hyper
    B = args.batch
    ctx = gp.Context(0)
    ctx.set_option("split_f16", int(args.split_f16))
    ps = ctx.assemble(torch.as_tensor(w.X, dtype=torch.float64, device="cuda"), hp.core_radius)
    rng = np.random.default_rng(7)
    tried = ps.autotune([synth_perturb(rng, hp) for _ in range(B)], reps=1)
    best = min(tried, key=lambda t: t["ms"])
    ps.set_blocking(best["group_blocks"], best["group_tile_n"])
    ev = mcmc.GpEvaluator(ctx, ps, B, gp.GP_MIXED)
    bounds = mcmc.Bounds(r0=(1e-3, 2.0 * float(hp.core_radius.max())), r=(0.02, 0.6), h=(-0.1, 1.1))
    s = mcmc.BlockMCMC(ev, w.resid, hp, B, seed=11, bounds=bounds)
    s.run(args.warmup)
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    calls0, fac0 = ev.calls, ev.factorizations
    t0 = time.perf_counter()
    s.run(args.steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    clocks = clk.stop()
    evals = (ev.calls - calls0) * B
    acc = {k: v / float(B * s.iterations) for k, v in s.accept_counts.items()}
    line = {"metric": "MCMC iterations/s (App. C blocks, lockstep chains)", "value": args.steps / dt,
            "unit": "iterations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "dtype": "f16+f64" if args.split_f16 else "tf32+f64",
            "data": "synthetic (seeded; the 200k-point batched workload)",
            "config": {"workload": "mcmc_200k", "n": int(w.X.shape[0]), "chains": B,
                       "blocking": {"group_blocks": best["group_blocks"], "group_tile_n": best["group_tile_n"]}},
            "loglik_evals_per_s": evals / dt,
            "factorizations_per_iteration": (ev.factorizations - fac0) / args.steps,
            "acceptance": acc, "clocks": clocks}
    print(json.dumps(line))
    ev.free()
    ps.free()


def synth_perturb(rng, hp):
    from paper_2411_05869_gb300 import synth
    return synth.perturb(rng, hp, 0.1)


# ------------------------------------------------------------------------------------------------ serving leg

def run_serving(args):
    """The serving mix: 20 cached point sets (n log-uniform in [5k, 500k], ~60 nnz/row, 16 bumps), requests of
    70 % log-likelihood and 30 % predictive mean (m uniform in 1000..50000 test points), Poisson arrivals at
    rates swept around the measured saturation rate, through the library's request server."""
    import torch
    from paper_2411_05869_gb300 import gp, synth
    sets = synth.serving_pointsets(count=args.serve_sets)
    srv_budget = int(args.serve_budget_gb * 1e9)
    rng = np.random.default_rng(4242)

    def requests(count, prec):
        out = []
        for _ in range(count):
            i = int(rng.integers(len(sets)))
            th = synth.perturb(rng, sets[i].hyper, 0.1)
            m = int(rng.integers(1000, 50001)) if rng.random() < 0.3 else 0
            out.append((i, th, m, prec))
        return out

    def run(srv, ids, resid, reqs, rate):
        """Submit at Poisson arrival times (rate None: all at once); per-request latency from submission."""
        keep, lat = {}, []
        t0 = time.perf_counter()
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs))) if rate else np.zeros(len(reqs))
        for (i, th, m, prec), ta in zip(reqs, arrivals):
            wait = t0 + ta - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            if m:
                xt = torch.rand(m, 3, dtype=torch.float64, device="cuda")
                out = torch.empty(m, dtype=torch.float64, device="cuda")
                rid = srv.submit(ids[i], th, resid[i], out, prec, Xtest=xt)
                keep[rid] = (xt, out)
            else:
                out = torch.empty(1, dtype=torch.float64, device="cuda")
                rid = srv.submit(ids[i], th, resid[i], out, prec)
                keep[rid] = (out,)
        srv.wait(0.0)
        done = srv.poll(4096)
        bad = sum(1 for c in done if c["status"] != 0)
        lat = np.array([c["t_done"] - c["t_submit"] for c in done])
        span = max(c["t_done"] for c in done) - min(c["t_submit"] for c in done)
        return {"requests": len(done), "failed": bad, "req_per_s": len(done) / span,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3)}

    result = {}
    for prec, name in ((gp.GP_MIXED, "mixed"), (gp.GP_FP64, "fp64")):
        if name == "fp64" and args.serve_fp64_requests <= 0:
            continue
        srv = gp.Server(0, slots=args.serve_slots, mem_budget_bytes=srv_budget)
        ids = [srv.add_pointset(torch.as_tensor(w.X, device="cuda"), w.hyper.core_radius) for w in sets]
        resid = [torch.as_tensor(w.resid, device="cuda") for w in sets]
        count = args.serve_requests if name == "mixed" else args.serve_fp64_requests
        run(srv, ids, resid, requests(min(count, 2 * len(sets)), prec), None)   # warm the factor cache
        sat = run(srv, ids, resid, requests(count, prec), None)
        sweep = {"saturation": sat}
        if name == "mixed":
            for f in args.serve_rates:
                sweep[f"{f:g}x"] = run(srv, ids, resid, requests(count, prec), f * sat["req_per_s"])
        sweep["server"] = srv.stats()
        result[name] = sweep
        srv.close()
    ns = [int(w.X.shape[0]) for w in sets]
    line = {"metric": "serving mix requests/s and p50/p99 latency (mixed vs FP64)",
            "value": result["mixed"]["saturation"]["req_per_s"], "unit": "requests/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic",
            "dtype": "f16+f64 (the server's contexts take the library's default operand split)",
            "config": {"workload": "serving", "sets": len(sets), "n_min": min(ns), "n_max": max(ns),
                       "slots": args.serve_slots, "budget_gb": args.serve_budget_gb,
                       "mix": "70% loglik, 30% predict (m ~ U{1000..50000})"},
            "serving": result}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=os.environ.get("GP_BENCH_WORKLOAD", "station_1.2M"))
    ap.add_argument("--precision", default=os.environ.get("GP_BENCH_PRECISION", "mixed"), choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=3, help="mixed runs: timed FP64 comparison steps (0: none)")
    ap.add_argument("--fp64-proposals", type=int, default=8, help="batched runs: proposals compared with FP64")
    ap.add_argument("--batch", type=int, default=0,
                    help="proposals per step (default: 64 for batched_200k, 16 chains for mcmc_200k, else 1)")
    ap.add_argument("--autotune", type=int, default=-1, help="1/0: tune the update blocking first (default: "
                                                              "on in mixed precision)")
    ap.add_argument("--blocking", default="", help="G,TN: fixed update blocking of mixed runs (no autotuner)")
    ap.add_argument("--diag-fp32", action="store_true",
                    help="mixed runs: factor the 64 x 64 diagonal blocks in FP32 (default FP64)")
    ap.add_argument("--split-f16", type=int, default=int(os.environ.get("GP_BENCH_SPLIT_F16", "1")), choices=[0, 1],
                    help="mixed runs: 1 = FP16 operand pairs for the tensor-core updates (GP_OPT_SPLIT_F16), "
                         "0 = TF32 pairs")
    ap.add_argument("--other-split", type=int, default=1, help="mixed runs at B = 1: also time the other operand "
                                                                 "split (1) or not (0)")
    ap.add_argument("--oracle-points", type=int, default=30_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--var-points", type=int, default=4096, help="test points of the predictive-variance timing")
    ap.add_argument("--iterative-probes", type=int, default=32,
                    help="probes of the paper's iterative comparison (stochastic Lanczos + MINRES; 0: skip)")
    ap.add_argument("--iterative-steps", type=int, default=30, help="Lanczos steps per probe")
    ap.add_argument("--oracle-threads", type=int, default=0, help="host threads of the threaded oracle leg "
                                                                   "(0: all cores)")
    ap.add_argument("--subwindow-parity", type=int, default=1, help="1: the GPU path on the oracle's sub-window "
                                                                    "against the oracle (FP64 and mixed)")
    ap.add_argument("--batch-leg", type=int, default=-1, help="mixed runs at B = 1: also time this many settings "
                    "per factorization (default 3 on station_1.2M, else 0)")
    ap.add_argument("--batch-leg-steps", type=int, default=3)
    ap.add_argument("--batch-leg-budget-gb", type=float, default=180.0, help="device memory the batched leg's "
                    "factor may take (the leg's B shrinks to fit)")
    ap.add_argument("--serve-sets", type=int, default=20)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=200.0)
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-fp64-requests", type=int, default=12)
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[0.25, 0.5, 1.0, 1.5])
    args = ap.parse_args()
    if args.batch <= 0:
        args.batch = {"batched_200k": 64, "mcmc_200k": 16}.get(args.workload, 1)
    if args.batch_leg < 0:
        args.batch_leg = 3 if args.workload == "station_1.2M" else 0
    if args.autotune < 0:   # the library's autotuner picks the update blocking of mixed runs (compact core)
        args.autotune = 1 if args.precision == "mixed" and args.workload != "noncompact_50k" else 0

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    peaks, peak_src = load_peaks()
    metric = "exact GP loglik evals/sec"

    if args.impl == "reference":
        if rank != 0:
            return
        w = make_workload(args.workload)
        full_flops = float(os.environ.get("GP_BENCH_FULL_FLOPS", 0.0)) or _full_flops_hint(args.workload)
        leg = OracleLeg(w, args.oracle_points, full_flops)
        from paper_2411_05869_gb300 import synth
        rng = np.random.default_rng(1234)
        cpu = host_cpu()
        thr = max(1, args.oracle_threads or cpu["nproc"] or 1)
        ts = []   # per step: `thr` evaluations of the sample, one per host thread
        for k in range(max(args.warmup, 0) + args.steps):
            dt = leg.step_threads([synth.perturb(rng, w.hyper, 0.05) for _ in range(thr)], thr)
            if k >= args.warmup:
                ts.append(dt)
        t_step = float(np.mean(ts)) * leg.scale          # projected wall time of thr full evaluations
        value = thr / t_step
        line = {"impl": "reference", "metric": metric, "value": value, "unit": "evals/s", "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3 / thr,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_config(w, args.workload, "fp64"),
                "latency_ms": {"p50": float(np.percentile(ts, 50)) * leg.scale * 1e3,
                               "p99": float(np.percentile(ts, 99)) * leg.scale * 1e3},
                "cpu_baseline": {"value": value, "unit": "evals/s", "cores": thr, "kind": "oracle",
                                 "cpu": cpu,
                                 "sample": leg.describe(float(np.mean(ts))) +
                                           f"; {thr} settings per step, one per host thread"},
                "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.workload == "serving":
        if rank == 0:
            run_serving(args)
        return
    if args.workload == "mcmc_200k":
        if rank == 0:
            run_mcmc(args)
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    res = run_gpu(args, rank, world, local_rank)
    tot_s = res["total_ms"] / 1e3
    if world > 1:
        tot_s = max_over_ranks(tot_s, f"cuda:{local_rank}")
    if rank != 0:
        return
    value = whole_job_rate(args.steps * res["Bc"] * res["nchunk"], world, tot_s)
    per = np.array(res["per"])
    info = res["info"]
    prof = res["prof"]
    a7 = ["extend_add", "front_small", "potrf", "trsm", "update", "update_left"]
    t_a7 = sum(prof[k][0] for k in a7)
    flops = info["flops"]
    f16 = args.precision == "mixed" and args.split_f16 == 1
    if f16:   # FP16 MMAs: the dense FP16 rate is the BF16 rate
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        bound, peak_note = "tensor", f"FP16 = {peak_src} bf16 sustained (the same nominal dense rate; of {peak_src})"
    elif args.precision == "mixed":   # the kernel runs inside a seconds-long step: the sustained figure applies
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * NOMINAL_TF32_OVER_BF16
        bound, peak_note = "tensor", f"TF32 = {peak_src} bf16 sustained x nominal 1.1/2.25 (of {peak_src})"
    else:
        peak = MEASURED_FP64_TFLOPS
        bound, peak_note = "alu", "FP64 FMA throughput measured on this pool"
    # the dominant kernel among the classes with a flop count (the tensor-core updates, POTRF, TRSM)
    dom = max(["potrf", "trsm", "update", "update_left"], key=lambda k: prof[k][0])
    d_ms, d_n, d_fl_front = prof[dom]
    # The classes count the flops of the relaxed fronts (explicit zeros included); the algorithmic work is
    # sum_j eta_j^2 over the exact column counts, so each class's count is scaled by the ratio of the two totals.
    front_total = sum(prof[k][2] for k in ("potrf", "trsm", "update", "update_left"))
    alg_ratio = (res["Bc"] * res["nchunk"] * flops / front_total) if front_total > 0 else 1.0
    d_fl = d_fl_front * alg_ratio
    achieved = d_fl / (d_ms * 1e-3) / 1e12 if d_ms > 0 else 0.0
    tkey = (args.workload, dom) + _blocking_of(res) + (("f16",) if f16 else ())
    kernels = {k: {"ms": round(v[0], 3), "launches": v[1], "useful_tflops": (round(v[2] / (v[0] * 1e-3) / 1e12, 3)
                                                                            if v[0] > 0 and v[2] > 0 else None)}
               for k, v in prof.items()}
    line = {
        "metric": metric, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(tot_s * 1e3 / args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else ("f16+f64" if f16 else "tf32+f64"),
        "data": "synthetic (seeded; shapes of the paper's space-time temperature workload)",
        "config": workload_config(res["w"], args.workload, args.precision,
                                  {"parallelism": f"replicas{world}", "B": res["B"],
                                   "operand_split": ("fp16 pairs x 2^k (3 kind::f16 MMAs per step)" if f16 else
                                                     "tf32 pairs (3 kind::tf32 MMAs per step)")
                                   if args.precision == "mixed" else None,
                                   "evaluations_per_step": res["Bc"] * res["nchunk"],
                                   "proposals_per_factorization": res["Bc"], "factorizations_per_step": res["nchunk"],
                                   "nnz": info["nnz"], "nnzL": info["nnzL"],
                                   "supernodes": info["nsuper"], "levels": info["nlevels"],
                                   "max_front": info["max_front"], "assemble_s": round(res["t_assemble"], 3)}),
        "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
        "roofline": {"kernel": (KERNEL_OF_CLASS_MIXED if args.precision == "mixed" else KERNEL_OF_CLASS_FP64).get(dom, dom),
                     "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None, "traffic": _TRAFFIC.get(tkey),
                     "launches_per_step": d_n, "avg_launch_ms": d_ms / max(d_n, 1),
                     "algorithmic": f"algorithmic flops of the class per step = {d_fl:.4g} (per launch "
                                    f"{d_fl / max(d_n, 1):.4g}): its relaxed-front flops {d_fl_front:.4g} x "
                                    f"{alg_ratio:.4f} (sum_j eta_j^2 = {flops:.4g} per proposal over the relaxed-front "
                                    f"flops of all A7 classes)",
                     "peak_source": peak_note,
                     "traffic_source": (("ncu dram__bytes_read.sum + dram__bytes_write.sum of all the class's launches "
                                         "in a factorization of station_120k at this blocking (L2 cold at each launch "
                                         "under ncu), " + ("per launch" if args.workload == "station_120k" else
                                         "as bytes per algorithmic flop times this workload's flops per launch "
                                         "(an estimate: traffic taken in proportion to the work)")))
                                       if _TRAFFIC.get(tkey) else None,
                     "traffic_before_wind_down": _TRAFFIC_EARLIER.get(tkey),
                     "a7_total": {"ms": t_a7, "proposals": res["Bc"] * res["nchunk"],
                                  "achieved": res["Bc"] * res["nchunk"] * flops / (t_a7 * 1e-3) / 1e12 if t_a7 > 0 else None}},
        "kernels": kernels,
        "e2e": {"value": res["e2e_steps"] * res["Bc"] * res["nchunk"] / res["e2e_s"], "unit": "evals/s", "h2d_bytes_per_step": res["h2d"],
                "d2h_bytes_per_step": res["d2h"]},
        "gpu_launches": int(res["launches"]),
        "clocks": res["clk"],
        "loglik_last": res["ll"],
    }
    if "fp64" in res:
        line["fp64"] = res["fp64"]
    if "other_split" in res:
        line["other_split"] = res["other_split"]
    if "batched" in res:
        line["batched"] = res["batched"]
    if res.get("predict"):
        line["predict"] = res["predict"]
    if res.get("variance"):
        line["predict_variance"] = res["variance"]
    if res.get("iterative"):
        line["iterative_comparison"] = res["iterative"]
    if res.get("autotune"):
        line["autotune"] = res["autotune"]
    if world == 1 and not args.no_cpu_baseline:
        cpu = host_cpu()
        try:
            leg = OracleLeg(res["w"], args.oracle_points, flops)
            dt = leg.step(res["w"].hyper)
            line["cpu_baseline"] = {"value": 1.0 / (dt * leg.scale), "unit": "evals/s", "cores": 1,
                                    "kind": "oracle", "cpu": cpu, "sample": leg.describe(dt)}
            thr = max(1, args.oracle_threads or cpu["nproc"] or 1)
            if thr > 1:
                from paper_2411_05869_gb300 import synth
                rng = np.random.default_rng(99)
                dtt = leg.step_threads([synth.perturb(rng, res["w"].hyper, 0.05) for _ in range(thr)], thr)
                line["cpu_baseline_threads"] = {"value": thr / (dtt * leg.scale), "unit": "evals/s", "cores": thr,
                                                "kind": "oracle", "sample": f"{thr} settings at once, one per host "
                                                f"thread, on the same sample ({dtt:.2f} s wall)"}
        except Exception as e:  # the baseline is reported, never required
            line["cpu_baseline"] = {"value": None, "unit": "evals/s", "cores": 1, "kind": "oracle", "cpu": cpu,
                                    "sample": f"failed: {e}"}
            leg = None
        if leg is not None and args.subwindow_parity:
            from paper_2411_05869_gb300 import gp
            ctx = res["ctx"]
            try:
                line["subwindow_parity"] = subwindow_parity(ctx, leg, res["w"].hyper,
                                                            [("fp64", gp.GP_FP64), ("mixed", gp.GP_MIXED)])
            except Exception as e:
                line["subwindow_parity"] = {"failed": str(e)}
    print(json.dumps(line))


# the kernel behind each timed class
KERNEL_OF_CLASS_MIXED = {"update": "k_update_ws<256, pair> (group-end updates: 256 x 256 CTA-pair tcgen05 MMAs)",
                         "update_left": "k_update_ws<128> (left-looking updates of block-column pairs, 128 x 128 tiles)",
                         "potrf": "k_potrf_pair (FP32 elimination with inverses) + k_potrf_tiles64 (FP64 L_11)",
                         "trsm": "k_trsm32_pair", "extend_add": "k_extend_add32"}
KERNEL_OF_CLASS_FP64 = {"update": "k_update (FP64 trailing updates)", "potrf": "k_potrf", "trsm": "k_trsm",
                        "extend_add": "k_extend_add"}

# DRAM bytes per launch of the dominant kernel by (workload, class, update blocking[, operand split]), from ncu
# captures of the current kernel; None where there is none. FP16 pairs, station_120k: all 79 group-end launches of
# a factorization at (32, 256) read and wrote 1.8894e9 bytes for 2.612e11 algorithmic flops (0.00723 bytes per
# flop). station_1.2M is too large for a multi-metric capture: its figure is that rate times the 1.901e11
# algorithmic flops of an average launch there (an estimate that assumes traffic in proportion to the work). TF32
# pairs at (16, 256): 2.924e9 bytes over 83 launches for 3.03e11 flops at 120k, 1.711e11 flops per launch at 1.2M.
_TRAFFIC = {("station_120k", "update", 32, 256, "f16"): 1.8894e9 / 79,
            ("station_1.2M", "update", 32, 256, "f16"): 1.8894e9 / 2.612e11 * 1.901e11,
            ("station_120k", "update", 16, 256): 2.924e9 / 83,
            ("station_1.2M", "update", 16, 256): 2.924e9 / 3.03e11 * 1.711e11}
_TRAFFIC_EARLIER = {("station_1.2M", "update", 16, 256): 2.712e9}


def _blocking_of(res):
    ch = (res.get("autotune") or {}).get("chosen") or {}
    return (ch.get("group_blocks"), ch.get("group_tile_n"))


def _full_flops_hint(name):
    return {"station_1.2M": 4.47e13, "spacetime_100k": 1.07e11, "batched_200k": 8.67e11}.get(name, 0.0)


if __name__ == "__main__":
    main()
