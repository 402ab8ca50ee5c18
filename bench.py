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

MEASURED_FP64_TFLOPS = 1.011   # FP64 FMA throughput measured on this GB300 pool
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def make_workload(name: str):
    from paper_2411_05869_gb300 import synth
    if name == "station_1.2M":
        return synth.config(5, with_test=False)
    if name == "station_120k":   # the same field over the first 24 days: a profiling-size case
        return synth.station_spacetime(nsites=5000, ndays=24, with_test=False)
    if name == "spacetime_100k":
        return synth.config(2, m=0)
    if name == "batched_200k":
        return synth.uniform_spacetime(200_000, 0, 80.0, 8, seed=synth.SEED_BASE + 3, name="spacetime_200k")
    if name == "spatial_2k":
        return synth.spatial_2d(n=2000, m=0, seed=synth.SEED_BASE + 1)
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
        self.rp, self.col = oracle.pattern(self.X, self.hp.core_radius)
        self.perm = oracle.fill_order(self.X, self.hp.core_radius, self.rp, self.col)
        sym = oracle.symbolic(self.rp, self.col, self.perm, want_rows=False)
        self.t_setup = time.perf_counter() - t0
        self.sample_flops = float((sym["eta"].astype(np.float64) ** 2).sum())
        self.scale = max(full_flops / self.sample_flops, 1.0) if full_flops > 0 else 1.0

    def step(self, theta) -> float:
        t0 = time.perf_counter()
        self.oracle.sparse_loglik(theta, self.X, self.rp, self.col, self.perm, self.r)
        return time.perf_counter() - t0

    def describe(self, t_eval: float) -> str:
        return (f"{self.desc}; oracle sparse loglik {t_eval:.2f} s per evaluation ({self.sample_flops:.3g} flops), "
                f"projected to the full workload by the flop ratio x{self.scale:.4g}")


# ------------------------------------------------------------------------------------------------ GPU leg

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
    with torch.cuda.stream(stream):
        X = torch.as_tensor(w.X, dtype=torch.float64, device=dev)
        resid = torch.as_tensor(w.resid, dtype=torch.float64, device=dev)
    stream.synchronize()
    t0 = time.perf_counter()
    ps = ctx.assemble(X, hp.core_radius)
    t_assemble = time.perf_counter() - t0
    info = ps.info()
    rng = np.random.default_rng(1234 + rank)
    from paper_2411_05869_gb300 import synth
    thetas = [synth.perturb(rng, hp, 0.05) for _ in range(max(args.steps, 1) + args.warmup + 8)]
    f = ctx.factor(ps, [hp], prec)
    out = torch.empty(1, dtype=torch.float64, device=dev)

    def step(i):
        f.update([thetas[i % len(thetas)]])
        f.loglik(resid, out=out)

    # warm-up
    for i in range(args.warmup):
        step(i)
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
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
    clk = clocks.stop()
    launches = ctx.launches() - launches0
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[args.steps])
    ll_last = float(out.cpu()[0])

    # end to end through the public API from host buffers: H2D of r from pinned memory, theta structs from
    # the host, D2H of the log-likelihood, every step
    r_host = torch.from_numpy(np.ascontiguousarray(w.resid)).pin_memory()
    out_host = torch.empty(1, dtype=torch.float64).pin_memory()
    r_dev = torch.empty_like(resid)
    e2e_steps = max(1, min(args.steps, 5))
    stream.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(e2e_steps):
            r_dev.copy_(r_host, non_blocking=True)
            f.update([thetas[k]])
            f.loglik(r_dev, out=out)
            out_host.copy_(out, non_blocking=True)
            stream.synchronize()
    e2e_s = time.perf_counter() - t0

    # per-kernel-class profile of one more step (not part of the timed region)
    ctx.profile(True)
    step(0)
    stream.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)

    res = dict(total_ms=total_ms, per=per, launches=launches, clk=clk, info=info, t_assemble=t_assemble,
               e2e_s=e2e_s, e2e_steps=e2e_steps, n=int(w.X.shape[0]), prof=prof, ll=ll_last,
               h2d=int(w.resid.nbytes), d2h=8, w=w)
    # FP64 comparison (mixed runs only): one evaluation of the same setting through the FP64 path, timed from
    # the call that creates (allocates and factors) the FP64 factor to its log-likelihood
    if prec == gp.GP_MIXED and args.fp64_steps > 0:
        th = thetas[0]
        f.update([th])
        f.loglik(resid, out=out)
        ll_mixed = float(out.cpu()[0])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            f64 = ctx.factor(ps, [th], gp.GP_FP64)
            f64.loglik(resid, out=out)
            e1.record(stream)
        stream.synchronize()
        ll64 = float(out.cpu()[0])
        res["fp64"] = {"ms_per_step": e0.elapsed_time(e1), "evals_per_s": 1e3 / e0.elapsed_time(e1),
                       "loglik": ll64, "mixed_loglik": ll_mixed,
                       "mixed_rel_diff": abs(ll_mixed - ll64) / abs(ll64),
                       "note": "one evaluation of the FP64 path (creation, first factorization and loglik)"}
        f64.free()
    f.free()
    ps.free()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=os.environ.get("GP_BENCH_WORKLOAD", "station_1.2M"))
    ap.add_argument("--precision", default=os.environ.get("GP_BENCH_PRECISION", "mixed"), choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--oracle-points", type=int, default=30_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

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
        ts = []
        for k in range(max(args.warmup, 0) + args.steps):
            dt = leg.step(synth.perturb(rng, w.hyper, 0.05))
            if k >= args.warmup:
                ts.append(dt)
        t_eval = float(np.mean(ts)) * leg.scale
        value = 1.0 / t_eval
        line = {"impl": "reference", "metric": metric, "value": value, "unit": "evals/s", "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_eval * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(w, args.workload, "fp64"),
                "latency_ms": {"p50": float(np.percentile(ts, 50)) * leg.scale * 1e3,
                               "p99": float(np.percentile(ts, 99)) * leg.scale * 1e3},
                "cpu_baseline": {"value": value, "unit": "evals/s", "cores": 1, "kind": "oracle",
                                 "sample": leg.describe(float(np.mean(ts)))},
                "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    res = run_gpu(args, rank, world, local_rank)
    tot_s = res["total_ms"] / 1e3
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([tot_s], dtype=torch.float64, device=f"cuda:{local_rank}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_s = float(t.item())
    if rank != 0:
        return
    value = args.steps * world / tot_s
    per = np.array(res["per"])
    info = res["info"]
    prof = res["prof"]
    a7 = ["extend_add", "front_small", "potrf", "trsm", "update"]
    t_a7 = sum(prof[k][0] for k in a7)
    flops = info["flops"]
    if args.precision == "mixed":
        peak = peaks["bf16_tflops"] * NOMINAL_TF32_OVER_BF16
        bound, peak_note = "tensor", f"TF32 = {peak_src} bf16 burst x nominal 1.1/2.25 (of {peak_src})"
    else:
        peak = MEASURED_FP64_TFLOPS
        bound, peak_note = "alu", "FP64 FMA throughput measured on this pool"
    dom = max(a7, key=lambda k: prof[k][0])
    d_ms, d_n, d_fl = prof[dom]
    achieved = d_fl / (d_ms * 1e-3) / 1e12 if d_ms > 0 else 0.0
    kernels = {k: {"ms": round(v[0], 3), "launches": v[1], "useful_tflops": (round(v[2] / (v[0] * 1e-3) / 1e12, 3)
                                                                            if v[0] > 0 and v[2] > 0 else None)}
               for k, v in prof.items()}
    line = {
        "metric": metric, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(tot_s * 1e3 / args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "tf32+f64",
        "data": "synthetic (seeded; shapes of the paper's space-time temperature workload)",
        "config": workload_config(res["w"], args.workload, args.precision,
                                  {"parallelism": f"replicas{world}", "nnz": info["nnz"], "nnzL": info["nnzL"],
                                   "supernodes": info["nsuper"], "levels": info["nlevels"],
                                   "max_front": info["max_front"], "assemble_s": round(res["t_assemble"], 3)}),
        "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
        "roofline": {"kernel": {"update": "k_update_ws (tensor-core trailing updates)"}.get(dom, dom),
                     "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None, "traffic": _TRAFFIC.get((args.workload, dom)),
                     "launches_per_step": d_n, "avg_launch_ms": d_ms / max(d_n, 1),
                     "algorithmic": f"useful flops of the class per step = {d_fl:.4g} (per launch "
                                    f"{d_fl / max(d_n, 1):.4g}); A7 total sum_j eta_j^2 = {flops:.4g}",
                     "peak_source": peak_note,
                     "a7_total": {"ms": t_a7, "achieved": flops / (t_a7 * 1e-3) / 1e12 if t_a7 > 0 else None}},
        "kernels": kernels,
        "e2e": {"value": res["e2e_steps"] / res["e2e_s"], "unit": "evals/s", "h2d_bytes_per_step": res["h2d"],
                "d2h_bytes_per_step": res["d2h"]},
        "gpu_launches": int(res["launches"]),
        "clocks": res["clk"],
        "loglik_last": res["ll"],
    }
    if "fp64" in res:
        line["fp64"] = res["fp64"]
    if world == 1 and not args.no_cpu_baseline:
        try:
            leg = OracleLeg(res["w"], args.oracle_points, flops)
            dt = leg.step(res["w"].hyper)
            line["cpu_baseline"] = {"value": 1.0 / (dt * leg.scale), "unit": "evals/s", "cores": 1,
                                    "kind": "oracle", "sample": leg.describe(dt)}
        except Exception as e:  # the baseline is reported, never required
            line["cpu_baseline"] = {"value": None, "unit": "evals/s", "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {e}"}
    print(json.dumps(line))


# DRAM bytes per launch of the dominant kernel, from ncu (profiles/), or None when the kernel changed since
_TRAFFIC = {("station_1.2M", "update"): 6.1e8}


def _full_flops_hint(name):
    return {"station_1.2M": 4.47e13, "spacetime_100k": 1.07e11, "batched_200k": 8.67e11}.get(name, 0.0)


if __name__ == "__main__":
    main()
