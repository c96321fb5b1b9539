#!/usr/bin/env python
"""Benchmark of the coupled LB + Oldroyd-B step: MLUPS and fraction of the HBM roofline.

Workload (default): the single-large-domain throughput case, a 512^3 periodic box with
1 % seeded Bernoulli obstacles, u ~ U(-1e-3, 1e-3), zero stress, beta = 0.5,
lambda = 1000, eta = 1/6.  One "step" is one time step of the whole coupled method over
the whole domain.  The state (~20 GB in FP32 storage) is far larger than L2, so no
flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent replica of
the workload (weak scaling; the method needs no collective for independent solves).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled LB+Oldroyd-B MLUPS (512^3 throughput workload)"
UNIT = "MLUPS"
HBM_FALLBACK_GBS = 6800.0
HBM_NOMINAL_GBS = 8000.0  # GB300 HBM3e, nominal

# Algorithmic bytes per cell update of the whole step: each PDF and stress value read
# once and written once, plus the flag byte (FP32 stress in the reduced-precision modes).
PDF_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}
REAL_BYTES = {"f64": 8, "f32": 4, "f16": 4, "bf16": 4}


def step_bytes(prec):
    return 19 * PDF_BYTES[prec] * 2 + 6 * REAL_BYTES[prec] * 2 + 1


def kernel_bytes(kind, prec):
    """Inputs + outputs each kernel must move per cell (its own I/O)."""
    pb, rb = PDF_BYTES[prec], REAL_BYTES[prec]
    if kind == "lb":  # f read + write, tau read (polymer force), u write, flag
        return 19 * pb * 2 + 6 * rb + 3 * rb + 1
    if kind == "fv":  # tau read, u read, tau write, flag
        return 6 * rb * 2 + 3 * rb + 1
    if kind == "fused":  # f read + write, tau read + write, u read + write, flag
        return 19 * pb * 2 + 6 * rb * 2 + 3 * rb * 2 + 1
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# ---------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: LBVE_CLOCKS_DIR if set, else the system temporary directory
        d = os.environ.get("LBVE_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"lbve_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------
# CPU oracle timing (baseline leg and the reference arm)
# ---------------------------------------------------------------------------------
def oracle_sample(side, seed=0):
    from oracle import oracle
    from paper_2009_12279_gb300 import workloads

    cfg = workloads.config_throughput(side, seed=seed)
    prm = dict(cfg["params"])
    prm["g"] = prm.pop("body_force")
    o = oracle.Oracle(cfg["shape"], **prm)
    o.set_flags(cfg["flags_fn"]())
    o.init_fields(u=cfg["u_fn"]())
    return o


def cores_used():
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    omp = os.environ.get("OMP_NUM_THREADS")
    return min(n, int(omp)) if omp else n


def oracle_rate(target_s, side):
    """(MLUPS, steps, seconds) of the oracle on a side^3 sample, about target_s of work."""
    o = oracle_sample(side)
    t0 = time.perf_counter()
    o.step(1)
    one = max(time.perf_counter() - t0, 1e-3)
    steps = max(1, int(target_s / one))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return side ** 3 * steps / dt / 1e6, steps, dt


def cpu_baseline(target_s=15.0, side=64):
    mlups, steps, dt = oracle_rate(target_s, side)
    out = {"value": mlups, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
           "sample": f"{side}^3 periodic box of the same workload (1% obstacles, random u), {steps} steps, FP64, "
                     f"{dt:.1f} s"}
    # the same oracle on one thread (a separate process with OMP_NUM_THREADS=1), 32^3 sample
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_rate(5.0, 32)))" % ROOT)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
        m1, steps1, dt1 = json.loads(r.stdout.strip().splitlines()[-1])
        out["single_thread"] = {"value": m1, "unit": UNIT, "cores": 1,
                                "sample": f"32^3 box of the same workload, {steps1} steps, {dt1:.1f} s"}
    except Exception as exc:  # reported, not fatal: the multi-core figure stands
        out["single_thread"] = {"error": str(exc)[:200]}
    # the plain-method channel (4 x 32 x 4, 20000 steps) in full
    try:
        from oracle import oracle
        from paper_2009_12279_gb300 import workloads

        cfg = workloads.config_channel()
        prm = dict(cfg["params"])
        prm["g"] = prm.pop("body_force")
        o = oracle.Oracle(cfg["shape"], **prm)
        o.set_flags(cfg["flags"])
        t0 = time.perf_counter()
        o.step(cfg["steps"])
        dt = time.perf_counter() - t0
        cells = cfg["shape"][0] * cfg["shape"][1] * cfg["shape"][2]
        out["channel_full"] = {"value": cells * cfg["steps"] / dt / 1e6, "unit": UNIT, "seconds": dt,
                               "sample": f"4x32x4 channel, {cfg['steps']} steps, FP64"}
    except Exception as exc:
        out["channel_full"] = {"error": str(exc)[:200]}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # each step: one time step of a bounded sample of the workload (whole run a few minutes)
    side = 64 if args.steps <= 400 else max(24, int((400 * 64 ** 3 / args.steps) ** (1 / 3)))
    o = oracle_sample(side)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = side ** 3 * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"throughput box sample {side}^3 (1% obstacles, random u, beta 0.5, lambda 1000)",
                       "cells": side ** 3},
            "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
                             "sample": f"{side}^3 periodic box of the throughput workload per step"},
            "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------
# finite-volume variants of the stress update (--fv-terms, --giesekus-alpha); the default is
# the method's own update
FV_EXTRA = {}


def build_solver(n, prec, schedule, stream, torch, nz=None):
    from paper_2009_12279_gb300 import Solver, lbve, workloads

    cfg = workloads.config_throughput(n, nz=nz)
    cfg["params"].update(FV_EXTRA)
    sched = {"auto": lbve.SCHED_AUTO, "split": lbve.SCHED_SPLIT, "fused": lbve.SCHED_FUSED}[schedule]
    s = Solver(cfg["shape"], precision=prec, schedule=sched, stream=stream, **cfg["params"])
    flags = cfg["flags_fn"]()
    cfg["fluid_cells"] = int((flags == 0).sum())
    s.set_geometry(flags)
    del flags
    # initial velocity drawn on the device (seeded) to keep host memory small
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    nx, ny, nzz = cfg["shape"]
    u = (torch.rand((3, nzz, ny, nx), generator=g, device="cuda", dtype=torch.float64) * 2.0 - 1.0) * 1e-3
    s.init_fields_device(0, u.data_ptr(), 0)
    torch.cuda.synchronize()
    del u
    return s, cfg


def time_device(s, steps, warmup, torch, dist, stream):
    s.step(warmup)
    s.synchronize()
    s.set_kernel_timing(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    kt = s.kernel_times()
    s.set_kernel_timing(False)
    return ms, kt


def time_e2e(n, prec, schedule, steps, torch, stream_obj):
    """Whole job through the public API with host buffers: create, geometry and initial
    velocity uploaded from pinned host memory, `steps` time steps, rho/u/tau read back to
    pinned host memory.  Returns MLUPS over the wall time of the job."""
    from paper_2009_12279_gb300 import Solver, lbve, workloads

    cfg = workloads.config_throughput(n)
    flags = torch.from_numpy(cfg["flags_fn"]()).pin_memory()
    g = torch.Generator()
    g.manual_seed(1)
    u = ((torch.rand((3, n, n, n), generator=g, dtype=torch.float64) * 2.0 - 1.0) * 1e-3).pin_memory()
    out_rho = torch.empty((n, n, n), dtype=torch.float64).pin_memory()
    out_u = torch.empty((3, n, n, n), dtype=torch.float64).pin_memory()
    out_tau = torch.empty((6, n, n, n), dtype=torch.float64).pin_memory()
    sched = {"auto": lbve.SCHED_AUTO, "split": lbve.SCHED_SPLIT, "fused": lbve.SCHED_FUSED}[schedule]
    torch.cuda.synchronize()
    phases = {}
    t0 = time.perf_counter()
    tp = t0

    def mark(name):
        nonlocal tp
        s.synchronize()
        now = time.perf_counter()
        phases[name] = now - tp
        tp = now

    s = Solver(cfg["shape"], precision=prec, schedule=sched, stream=stream_obj.cuda_stream, **cfg["params"])
    mark("create_s")
    s.set_geometry(flags.numpy())
    mark("geometry_s")
    s.init_fields_ptr(0, u.data_ptr(), 0)
    mark("upload_s")
    s.step(steps)
    mark("steps_s")
    s.read_fields_ptr(out_rho.data_ptr(), out_u.data_ptr(), out_tau.data_ptr())
    mark("read_back_s")
    dt = time.perf_counter() - t0
    s.close()
    h2d = flags.numel() + u.numel() * 8
    d2h = (out_rho.numel() + out_u.numel() + out_tau.numel()) * 8
    finite = bool(torch.isfinite(out_u).all())
    return {"value": n ** 3 * steps / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps, "wall_s": dt, "job": f"create + upload + {steps} steps + read-back",
            "phases": phases, "finite": finite}


def bench_serving(args, torch):
    """Bounded sample of the serving workload: batched BF16 pool vs one-at-a-time FP32."""
    import numpy as np

    from paper_2009_12279_gb300 import lbve, serve

    stream = torch.cuda.Stream()
    kw = dict(max_steps_cap=args.serving_cap)
    reqs0 = serve.make_requests(args.serving_requests, seed=0, mean_interarrival=0.0, **kw)
    polish = "f32" if args.serving_polish else None
    # the one-at-a-time FP32 baseline runs on the first serving_solo requests (all by default)
    n_solo = args.serving_solo if args.serving_solo > 0 else len(reqs0)
    # tile autotuning (outside the timed runs): one solve per domain width of the stream
    # in a scratch pool; the recorded choices apply to every pool admitted to later
    tuning = {}
    for prec in ("bf16", "f32"):
        t0 = time.perf_counter()
        pool = lbve.Pool(prec, budget_bytes=int(args.serving_budget_gb * 1e9), stream=stream.cuda_stream)
        seen, scratch = set(), []
        for r in reqs0:
            if r.shape[0] in seen:
                continue
            seen.add(r.shape[0])
            sv = serve.build_solver(r, prec, stream.cuda_stream)
            pool.admit(sv)
            scratch.append(sv)
        res = pool.autotune(steps=10)
        pool.close()
        for sv in scratch:
            sv.close()
        torch.cuda.synchronize()
        res["tuning_s"] = time.perf_counter() - t0
        tuning[prec] = res
    # throughput mode (all requests waiting at t = 0)
    t0 = time.perf_counter()
    solo, fsolo = serve.run_one_at_a_time(reqs0[:n_solo], precision="f32", stream=stream.cuda_stream,
                                          keep_fields=True)
    torch.cuda.synchronize()
    wall_solo = time.perf_counter() - t0
    keep = {r.rid for r in reqs0[:n_solo]}  # fields kept for the accuracy comparisons only
    # batched FP32: bitwise the same results as one at a time (equal accuracy)
    mix32, wall_mix32, stats32, same = [], float("nan"), {}, None
    if not args.serving_config5:
        srv = serve.Server("f32", budget_bytes=int(args.serving_budget_gb * 1e9), stream=stream.cuda_stream)
        t0 = time.perf_counter()
        mix32, fmix32 = srv.run(reqs0, keep_fields=keep)
        torch.cuda.synchronize()
        wall_mix32 = time.perf_counter() - t0
        stats32 = dict(srv.stats)
        srv.close()
        same = all(all(np.array_equal(a, b) for a, b in zip(fsolo[r], fmix32[r])) for r in fsolo if r in fmix32)
    srv = serve.Server("bf16", budget_bytes=int(args.serving_budget_gb * 1e9), stream=stream.cuda_stream,
                       polish=polish)
    t0 = time.perf_counter()
    mix, fmix = srv.run(reqs0, keep_fields=keep)
    torch.cuda.synchronize()
    wall_mix = time.perf_counter() - t0
    peak = srv.peak_bytes
    stats16 = dict(srv.stats)
    srv.close()
    # accuracy of the batched BF16 results against the FP32 one-at-a-time results
    errs = []
    for rid, fs in fsolo.items():
        if rid in fmix:
            u32, u16 = fs[1], fmix[rid][1]
            errs.append(float(np.linalg.norm(u16 - u32) / max(np.linalg.norm(u32), 1e-300)))
    if args.serving_config5:
        # the stated stream is long (solves of up to 50,000 steps): latencies are taken from
        # the throughput runs (every request arriving at t = 0, latency = completion time)
        mean_gap, wall_lat, wall_lat_solo = 0.0, wall_mix, wall_solo
        s_mix, s_solo = serve.summarize(mix, wall_mix), serve.summarize(solo, wall_solo)
    else:
        # latency under Poisson arrivals at 0.8 x the batched service time per solve
        mean_gap = 0.8 * wall_mix / max(len(reqs0), 1)
        reqs = serve.make_requests(args.serving_requests, seed=0, mean_interarrival=mean_gap, **kw)
        srv = serve.Server("bf16", budget_bytes=int(args.serving_budget_gb * 1e9), stream=stream.cuda_stream,
                           polish=polish)
        t0 = time.perf_counter()
        lat_mix, _ = srv.run(reqs)
        torch.cuda.synchronize()
        wall_lat = time.perf_counter() - t0
        srv.close()
        t0 = time.perf_counter()
        lat_solo, _ = serve.run_one_at_a_time(reqs[:n_solo], precision="f32", stream=stream.cuda_stream)
        torch.cuda.synchronize()
        wall_lat_solo = time.perf_counter() - t0
        s_mix, s_solo = serve.summarize(lat_mix, wall_lat), serve.summarize(lat_solo, wall_lat_solo)
    return {
        "requests": len(reqs0), "step_cap": args.serving_cap, "stop": "residual 1e-6 per step or cap",
        "polish": polish, "one_at_a_time_requests": n_solo,
        "batched_bf16": {"solves_per_s": len(mix) / wall_mix, "wall_s": wall_mix,
                         "p50_latency_s": s_mix["p50_latency_s"], "p99_latency_s": s_mix["p99_latency_s"],
                         "poisson_wall_s": wall_lat, "peak_device_bytes": peak, "phases": stats16,
                         "mlups": serve.summarize(mix, wall_mix)["mlups"]},
        "batched_f32": None if not mix32 else {
            "solves_per_s": len(mix32) / wall_mix32, "wall_s": wall_mix32,
            "bitwise_equal_to_one_at_a_time": bool(same), "phases": stats32,
            "mlups": serve.summarize(mix32, wall_mix32)["mlups"]},
        "one_at_a_time_f32": {"solves_per_s": len(solo) / wall_solo, "wall_s": wall_solo,
                              "p50_latency_s": s_solo["p50_latency_s"], "p99_latency_s": s_solo["p99_latency_s"],
                              "poisson_wall_s": wall_lat_solo, "mlups": serve.summarize(solo, wall_solo)["mlups"]},
        "speedup_solves_per_s": (len(mix) / wall_mix) / (len(solo) / wall_solo),
        "tile_autotune": tuning,
        "mean_interarrival_s": mean_gap,
        "bf16_vs_f32_u_rel_l2": {"median": float(np.median(errs)) if errs else None,
                                 "max": float(np.max(errs)) if errs else None},
        "statuses_bf16": {k: sum(r.status == k for r in mix) for k in ("converged", "capped", "unstable", "rejected")},
        "polished_bf16": stats16.get("polished", 0),
        "statuses_f32": {k: sum(r.status == k for r in solo) for k in ("converged", "capped", "unstable", "rejected")},
        "unstable_bf16": [(r.rid, r.kind) for r in mix if r.status == "unstable"],
    }


def profile_pool_steps(args):
    """Pool steps of the serving mix between cudaProfilerStart / Stop, for a launch list
    taken with `ncu --profile-from-start off`: the first args.serving_requests requests of
    the serving stream (all resident, BF16 storage), 200 untimed pool steps (graph
    capture), 200 timed ones, then args.profile_pool_steps profiled steps.  Prints the
    mean pool step time of the timed steps."""
    import numpy as np
    import torch

    from paper_2009_12279_gb300 import lbve, serve

    stream = torch.cuda.Stream()
    reqs = serve.make_requests(args.serving_requests, seed=0, mean_interarrival=0.0, max_steps_cap=args.serving_cap)
    pool = lbve.Pool("bf16", budget_bytes=int(args.serving_budget_gb * 1e9), stream=stream.cuda_stream)
    solvers = [serve.build_solver(r, "bf16", stream.cuda_stream) for r in reqs]
    for s in solvers:
        pool.admit(s)
    pool.step(200)  # captures the step graph of a 200-step call
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pool.step(200)  # replays it
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) / 200 * 1e3
    torch.cuda.profiler.start()
    pool.step(args.profile_pool_steps)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"pool_step_ms": ms, "members": len(solvers), "profiled_steps": args.profile_pool_steps,
                      "cells": int(sum(np.prod(r.shape) for r in reqs))}), flush=True)
    pool.close()
    for s in solvers:
        s.close()
    return 0


def run_ours(args):
    import torch

    from paper_2009_12279_gb300 import build

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        torch.cuda.set_device(local)
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    from paper_2009_12279_gb300 import lbve

    lbve.load()
    # CPU baseline first (rank 0, N=1 only), before the GPU work of the timed runs
    cpu = cpu_baseline() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None

    stream_obj = torch.cuda.current_stream()
    stream = stream_obj.cuda_stream
    n = args.n
    peak, peak_kind = measured_peaks()
    results = {}
    clocks = None
    for prec in args.precisions:
        s, cfg = build_solver(n, prec, args.schedule, stream, torch, nz=args.nz)
        tuned = None
        if args.schedule != "fused" and not args.no_autotune:
            # schedule autotuning on the solve's own steps (launch shapes do not change
            # results); these steps come before the warm-up and the timed region
            t0 = time.perf_counter()
            tuned = s.autotune(steps=4)
            tuned["tuning_s"] = time.perf_counter() - t0
        sampler = ClockSampler(local) if prec == args.precisions[0] else None
        if sampler:
            sampler.start()
        ms, kt = time_device(s, args.steps, args.warmup, torch, dist, stream_obj)
        if sampler:
            clocks = sampler.stop()
        health = s.reduce()
        lb_kernel = s.stream_collide_kernel
        s.close()
        del s
        torch.cuda.empty_cache()
        t = torch.tensor([ms], device="cuda")
        if dist:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
        cells = n * n * (args.nz or n)
        mlups = world * cells * args.steps / (ms_max * 1e-3) / 1e6
        fluid_fraction = cfg["fluid_cells"] / cells
        dom = max(kt.items(), key=lambda kv: kv[1][0])
        kind, (kms, klaunch) = dom
        kb = kernel_bytes(kind, prec)
        achieved = kb * cells * klaunch / (kms * 1e-3) / 1e9 if kb else None
        launches = sum(c for k, (_, c) in kt.items()) + kt.get("momentum_exchange", (0, 0))[1]
        results[prec] = {
            "mlups": mlups, "ms_per_step": ms_max / args.steps,
            "step_roofline_frac": mlups * 1e6 * step_bytes(prec) / (peak * 1e9),
            "step_roofline_frac_nominal": mlups * 1e6 * step_bytes(prec) / (HBM_NOMINAL_GBS * 1e9),
            "fluid_mlups": mlups * fluid_fraction,
            "step_bytes_per_cell": step_bytes(prec),
            "kernels": {k: {"avg_ms": v[0] / max(v[1], 1), "launches": v[1],
                            "achieved_gbs": (kernel_bytes(k, prec) * cells * v[1] / (v[0] * 1e-3) / 1e9)
                            if kernel_bytes(k, prec) else None} for k, v in kt.items()},
            "stream_collide": lb_kernel,
            "roofline": {"bound": "hbm", "kernel": "k_lb_rows" if kind == "lb" and lb_kernel == "rows" else f"k_{kind}",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": None,
                         "bytes_per_cell": kb, "peak_source": peak_kind},
            "gpu_launches": launches,
            "healthy": not health["bad"],
            "schedule_tuning": tuned,
        }
    serving = None
    if rank == 0 and not args.no_serving:
        serving = bench_serving(args, torch)
    e2e = None
    if not args.no_e2e:
        e2e = time_e2e(n, args.precisions[0], args.schedule, args.steps, torch, stream_obj)
    if rank == 0:
        main = results[args.precisions[0]]
        traffic = load_traffic(args.precisions[0], main["roofline"]["kernel"], args.schedule)
        main["roofline"]["traffic"] = traffic
        line = {
            "metric": METRIC, "value": main["mlups"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precisions[0] == "f64" else "f32",
            "data": "synthetic",
            "config": {"workload": (f"throughput {n}^3" if not args.nz else f"throughput {n}x{n}x{args.nz}") +
                                   " periodic, 1% Bernoulli obstacles, u~U(-1e-3,1e-3), "
                                   f"beta 0.5, lambda 1000, eta 1/6, {args.precisions[0]} PDF storage",
                       "cells": n * n * (args.nz or n), "schedule": args.schedule, "parallelism": f"replicas{world}",
                       **({"fv_variants": dict(FV_EXTRA)} if FV_EXTRA else {}),
                       "l2": "state larger than L2 (no flush needed)",
                       "schedule_tuning": main.get("schedule_tuning"),
                       "step_bytes_per_cell": main["step_bytes_per_cell"]},
            "roofline": main["roofline"],
            "step_roofline_frac": main["step_roofline_frac"],
            "step_roofline_frac_nominal": main["step_roofline_frac_nominal"],
            "fluid_mlups": main["fluid_mlups"],
            "gpu_launches": main["gpu_launches"],
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "serving": serving,
            "modes": {p: {k: v for k, v in r.items() if k != "roofline"} | {"roofline_frac": r["roofline"]["frac"]}
                      for p, r in results.items()},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# Sources whose kernels the traffic record was measured on; any change to them makes the
# record stale (traffic is then reported as null until it is captured again).
KERNEL_SOURCES = ("lbve_device.cuh", "lbve_kernels.cuh", "lbve_rows.cuh", "lbve_table.cuh", "lbve_launch.h")


def kernel_sources_sha():
    import hashlib

    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2009_12279_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def load_traffic(prec, kernel, schedule):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if it
    was captured on these kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        rec = d.get("kernels", {}).get(f"{kernel}:{prec}")
        if not rec or d.get("kernel_sources_sha256") != kernel_sources_sha():
            return None
        return rec["dram_bytes_per_launch_full_size"]
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=512, help="side of the cubic throughput domain")
    ap.add_argument("--nz", type=int, default=None,
                    help="z extent of the throughput domain (n x n x nz; profiling of small cases)")
    ap.add_argument("--precisions", default="f32,f16,bf16", help="PDF storage modes; the first one is the headline")
    ap.add_argument("--schedule", choices=["auto", "split", "fused"], default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="time the default schedule")
    ap.add_argument("--serving-requests", type=int, default=None,
                    help="requests of the serving stream (default 48; 2000 with --serving-config5)")
    ap.add_argument("--serving-cap", type=int, default=1000, help="step cap per solve in the serving sample")
    ap.add_argument("--serving-budget-gb", type=float, default=150.0)
    ap.add_argument("--serving-polish", action="store_true",
                    help="BF16 solves that reach the BF16 residual floor finish in an FP32 pool")
    ap.add_argument("--serving-solo", type=int, default=0,
                    help="run the one-at-a-time FP32 baseline on the first this many requests (0: all)")
    ap.add_argument("--serving-config5", action="store_true",
                    help="the serving configuration as stated: 2000 requests, cap min(10 lambda, 50000) steps, "
                         "residual 1e-6 (BF16 with FP32 polish; one-at-a-time FP32 on the first 100)")
    ap.add_argument("--fv-terms", type=int, default=0,
                    help="LBVE_FV_* bits of the throughput solve (0: flux and source, the method)")
    ap.add_argument("--profile-pool-steps", type=int, default=0,
                    help="only run this many pool steps of the serving mix under cudaProfilerStart/Stop")
    ap.add_argument("--giesekus-alpha", type=float, default=0.0,
                    help="Giesekus mobility of the throughput solve (0: Oldroyd-B, the method)")
    args = ap.parse_args()
    if args.serving_requests is None and not args.serving_config5:
        args.serving_requests = 48
    if args.serving_config5:
        args.serving_requests = args.serving_requests or 2000
        args.serving_cap, args.serving_polish = 50000, True
        args.serving_solo = args.serving_solo or 100
    args.precisions = [p.strip() for p in args.precisions.split(",") if p.strip()]
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.fv_terms:
        FV_EXTRA["fv_terms"] = args.fv_terms
    if args.giesekus_alpha:
        FV_EXTRA["giesekus_alpha"] = args.giesekus_alpha
    if args.profile_pool_steps:
        return profile_pool_steps(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
