#!/usr/bin/env python3
"""Benchmark of the GB300 SIP solver (libsip.so through its C ABI).

Workload: the 256^3 pressure-Poisson block (16.8 M cells, symmetric 7-point
matrix with one Dirichlet face, alpha = 0.92), seeded synthetic inputs.

A step is one sip_solve call on the factored plan: the right-hand side and
the initial guess are copied into the plane layout, SIP iterations run with
the device-side stop rule (rtol 1e-8, at most --iters iterations per step),
and x is copied back; x is reset to 0 before every step.  `value` is the
FP32-refined solver's SIP rate in MLUP/s (cells x FP32 SIP iterations / step
time, the FP64 residual/refinement passes included in the time); the plain
FP64 solver is measured the same way under "fp64".  The factorisation is
timed separately (factor_ms).  "time_to_1e-8" times full solves of both
solvers to the 1e-8 relative residual; "serving" measures the request server
(continuous batching, p50/p99 latency) against a serial plain-FP64 queue.

--impl reference times the CPU oracle (plain C, one thread) on a bounded
sample of the same workload: each step is one FP64 SIP iteration of the
256^3 block.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SIP MLUP/s & %HBM roofline, FP32-refined vs FP64; p50/p99 solve latency"

# Algorithmic bytes per cell per launch of each kernel kind (each array read or
# written once; neighbour values reused on chip).  Words of 8 B (FP64) or 4 B.
# The residual kernels' figures are for a symmetric A (four stored entries).
ALGO_BYTES = {
    "factor": 7 * 8 + 7 * 8,           # A in, LB LW LS 1/LP UN UE UT out
    "factor32": 7 * 8 + 7 * 4,         # A in (FP64), FP32 factors out
    "resid64": 4 * 8 + 3 * 8,          # AP AE AN AT b x in, r out
    "resid32": 4 * 4 + 3 * 4, "resid32_norm": 4 * 4 + 3 * 4,
    "resid64_r32": 4 * 8 + 2 * 8 + 4,  # AP AE AN AT b x in (FP64), r out (FP32)
    "fwd64": 6 * 8,                    # LB LW LS 1/LP r in, y out
    "bwd64": 6 * 8,                    # UE UN UT y x in, x out
    "fwd32": 6 * 4,
    "bwd32": 6 * 4,                    # UE UN UT y d in, d out
    "bwd32_x0": 5 * 4,                 # UE UN UT y in, d out
    "update64": 4 + 16,                # d in, x64 in/out (refinement update)
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=256, help="cube edge of the Poisson block")
    ap.add_argument("--iters", type=int, default=100,
                    help="max FP64 corrections (refined) / iterations (fp64) per step")
    ap.add_argument("--inner", type=int, default=8, help="FP32 iterations per FP64 correction (8: fastest to 1e-8 at 256^3 and on the 64-block mesh)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=3)
    ap.add_argument("--no-ttol", action="store_true", help="skip the time-to-1e-8 solves")
    ap.add_argument("--no-inner-sweep", action="store_true",
                    help="time-to-1e-8 of the refined form with the default inner count only (skip m = 1, 2, 8)")
    ap.add_argument("--small-solves", type=int, default=200, help="solves of the 32^3 latency measurement")
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests of the serving measurement (0: skip)")
    ap.add_argument("--serve-min-n", type=int, default=16, help="smallest cube edge of a served request")
    ap.add_argument("--serve-max-n", type=int, default=192, help="largest cube edge of a served request")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-sat", type=int, default=500,
                    help="requests of the saturation run (a prefix of the request list)")
    ap.add_argument("--serve-capacity-prefix", type=int, default=400,
                    help="requests served with arrivals at 0.8 x the serial FP64 capacity (a prefix; 0: skip)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-block batched-mesh measurement")
    ap.add_argument("--no-small", action="store_true", help="skip the 32^3 solve-latency measurement")
    ap.add_argument("--no-assembly", action="store_true", help="skip the pressure-correction assembly measurement")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 384^3 Peclet-10 block with FP32 coefficients (alpha 0.5 and 0.92)")
    ap.add_argument("--batched-iters", type=int, default=12,
                    help="corrections (refined) / iterations (fp64) timed on the batched mesh")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return out
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[2][q].lower().startswith("active")})
        out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(r[1] for r in rows), reasons=reasons,
                   samples=len(rows))
        return out


SWEEP_SOURCES = ("sip_sweeps.cuh", "sip_layout.h", "sip_k32.cu", "sip_k64.cu", "sip_resrow.cu")


def src_hash() -> str:
    """Hash of the sources that define the sweep kernels (their DRAM traffic
    counters stay valid while these files are unchanged)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1303_4538_gb300", "csrc")
    for f in SWEEP_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str, cells: int):
    """DRAM bytes of one launch over `cells` cells from the committed ncu
    summary (its bytes per captured cell: every array is touched once per
    launch, so the traffic grows in proportion to the cells), if the capture
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("src_hash") != src_hash():
        return None
    v = d.get("kernels", {}).get(kernel)
    if not isinstance(v, dict) or not v.get("captured_cells"):
        return None
    return int(round(v["captured_bytes"] / v["captured_cells"] * cells))


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ oracle
def host_cpu():
    """CPU model and core count of this host (for the oracle timing)."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu part", "hardware") and ":" in line:
                model = line.split(":", 1)[1].strip()
                if key == "model name":
                    break
    except OSError:
        pass
    parts = {"0xd4f": "Arm Neoverse V2 (Grace)", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}
    return {"model": parts.get(model, model), "nproc": os.cpu_count()}


# The paper's own figures for this path (CPU, FP64): context, not a target.
PAPER_CPU = {
    "hardware": "Intel Xeon X5650 (Westmere), 1 core, Intel Fortran 12.1",
    "resforward3d_MB_per_s": 7116, "backward3d_MB_per_s": 7025, "lu3d_MB_per_s": 4204,
    "resforward3d_ms_per_call": round(56.48e3 / 7500, 2),
    "source": "arXiv:1303.4538 Tables 1 and 4 (profile of test case I, implicit, serial)",
    "note": "no cell counts per call are given, so no MLUP/s; about 0.5 M cells per call at 7.1 GB/s would be "
            "60-70 MLUP/s (order of magnitude only)",
}


def cpu_baseline(blk, iters: int):
    import numpy as np
    import oracle
    n = blk.nx
    t0 = time.perf_counter()
    F = oracle.factor(n, n, n, blk.coefs, 0.92)
    tf = time.perf_counter() - t0
    x = np.zeros(blk.n)
    oracle.iterate(n, n, n, blk.coefs, F, blk.b, x)  # warm
    t0 = time.perf_counter()
    for _ in range(iters):
        oracle.iterate(n, n, n, blk.coefs, F, blk.b, x)
    dt = time.perf_counter() - t0
    return blk.n * iters / dt / 1e6, dt, tf


def run_reference(args):
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.destroy_process_group()
            return
    import numpy as np
    import oracle
    from paper_1303_4538_gb300 import workloads as W
    blk = W.poisson_256cube(args.n)
    n = blk.nx
    F = oracle.factor(n, n, n, blk.coefs, 0.92)
    x = np.zeros(blk.n)
    for _ in range(args.warmup):
        oracle.iterate(n, n, n, blk.coefs, F, blk.b, x)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.iterate(n, n, n, blk.coefs, F, blk.b, x)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = blk.n * args.steps / tot / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"poisson_{n}cube", "cells": blk.n, "alpha": 0.92,
                   "step": "one FP64 SIP iteration (residual, forward, backward, update, norm)"},
        "cpu_baseline": {"value": value, "unit": "MLUP/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} FP64 SIP iterations of the {n}^3 Poisson block, 1 thread",
                         "host": host_cpu()},
        "paper_cpu_context": PAPER_CPU,
        "e2e": {"value": value, "unit": "MLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------ GPU path
def reduce_over_ranks(dist, times_ms, counts, device):
    """Replicas: the job's time is the slowest rank's (MAX), its work the sum
    of all ranks' (SUM).  Returns (times, counts) as Python lists."""
    import torch
    t = torch.tensor([float(v) for v in times_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), c.tolist()


def run_gb300(args):
    import numpy as np
    import torch

    from paper_1303_4538_gb300 import build as B
    from paper_1303_4538_gb300 import sip
    from paper_1303_4538_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    sip.lib()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    blk = W.poisson_256cube(args.n)
    N = blk.n
    stream = torch.cuda.current_stream()
    ctx = sip.Context(local, stream.cuda_stream)
    A = [torch.from_numpy(c).cuda() for c in blk.coef_list()]
    b = torch.from_numpy(blk.b).cuda()
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    desc = sip.make_desc(blk.nx, blk.ny, blk.nz, [A[0], None, A[2], None, A[4], None, A[6]], b, x, symmetric=True)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # tile shapes from the autotuner (plan creation, untimed)
    opt_r = tuned_options(ctx, [desc], mode=sip.SIP_MODE_F32_REFINED, inner_iters=args.inner)
    opt_d = tuned_options(ctx, [desc], mode=sip.SIP_MODE_F64)
    torch.cuda.synchronize()
    e0.record(stream)
    plan_r = sip.Plan(ctx, [desc], opt_r)
    e1.record(stream)
    torch.cuda.synchronize()
    factor_ms_r = e0.elapsed_time(e1)
    e0.record(stream)
    plan_d = sip.Plan(ctx, [desc], opt_d)
    e1.record(stream)
    torch.cuda.synchronize()
    factor_ms_d = e0.elapsed_time(e1)
    # A stays allocated: the inner-count sweep of the time-to-1e-8 factors more plans from it

    def step(plan):
        # a fixed number of corrections (rtol 0: the stop rule never fires)
        x.zero_()
        return plan.solve(0.0, args.iters)

    def timed(plan, inner, K, prof=False):
        barrier()
        if prof:
            plan.profile(True)
            plan.profile_read(reset=True)
        l0 = plan.launches()
        e0.record(stream)
        its = 0
        for _ in range(K):
            it, rel, conv = step(plan)
            its += it
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        prof_d = plan.profile_read(reset=True) if prof else {}
        if prof:
            plan.profile(False)
        return ms, its * inner, plan.launches() - l0, prof_d

    for _ in range(args.warmup):
        step(plan_r)
        step(plan_d)
    clocks = ClockSampler(local)
    clocks.start()
    ms_r, lup_iters_r, launches_r, _ = timed(plan_r, args.inner, args.steps)
    ms_d, lup_iters_d, launches_d, _ = timed(plan_d, 1, args.steps)
    clk = clocks.stop()
    # per-kernel breakdown (CUDA events around every launch) in a separate
    # untimed step, so the event records do not enter the timed value
    _, _, _, prof_r = timed(plan_r, args.inner, 1, prof=True)
    _, _, _, prof_d = timed(plan_d, 1, 1, prof=True)

    # end-to-end through the public API with host buffers
    b_h = torch.from_numpy(blk.b).pin_memory()
    x0_h = torch.zeros(N, dtype=torch.float64).pin_memory()
    x_h = torch.empty(N, dtype=torch.float64).pin_memory()
    barrier()
    e0.record(stream)
    e2e_iters = 0
    for _ in range(args.steps):
        b.copy_(b_h, non_blocking=True)
        x.copy_(x0_h, non_blocking=True)
        it, rel, conv = plan_r.solve(1e-8, args.iters)
        e2e_iters += it * args.inner
        x_h.copy_(x, non_blocking=True)
    e1.record(stream)
    barrier()
    ms_e2e = e0.elapsed_time(e1)

    ttol = {}
    if not args.no_ttol:
        runs = [("f32_refined", plan_r, args.inner, False), ("f64", plan_d, 1, False)]
        # the refined form with other numbers of FP32 iterations per FP64 correction
        for m in (1, 2, 4, 8):
            if m != args.inner and not args.no_inner_sweep:
                om = sip.default_options(mode=sip.SIP_MODE_F32_REFINED, inner_iters=m,
                                         rows_per_thread=opt_r.rows_per_thread, tile_k=opt_r.tile_k,
                                         stages=opt_r.stages)
                runs.append((f"f32_refined_m{m}", sip.Plan(ctx, [desc], om), m, True))
        for name, plan, inner, own in runs:
            barrier()
            x.zero_()
            e0.record(stream)
            it, rel, conv = plan.solve(1e-8, 1_000_000)
            e1.record(stream)
            barrier()
            ttol[name] = {"seconds": e0.elapsed_time(e1) / 1e3, "iterations": it, "sip_iterations": it * inner,
                          "relres": rel, "converged": conv}
            if own:
                plan.close()

    def rates(ms, iters):
        return N * iters / (ms / 1e3) / 1e6

    val_r = rates(ms_r, lup_iters_r)
    val_d = rates(ms_d, lup_iters_d)
    val_e2e = rates(ms_e2e, e2e_iters)
    if dist:
        (ms_r, ms_d, ms_e2e), c = reduce_over_ranks(dist, [ms_r, ms_d, ms_e2e],
                                                    [lup_iters_r, lup_iters_d, e2e_iters], "cuda")
        val_r = N * c[0] / (ms_r / 1e3) / 1e6
        val_d = N * c[1] / (ms_d / 1e3) / 1e6
        val_e2e = N * c[2] / (ms_e2e / 1e3) / 1e6

    hbm, src = peaks()

    def roofline(prof):
        sweep = {k: v for k, v in prof.items() if k in ALGO_BYTES}
        if not sweep:
            return None
        k = max(sweep, key=lambda q: sweep[q][0])
        tot_ms, n = sweep[k]
        per_launch_s = tot_ms / n / 1e3
        ach = ALGO_BYTES[k] * N / per_launch_s / 1e9
        return {"bound": "hbm", "kernel": k, "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "traffic": load_traffic(k, N), "peak_source": src,
                "algo_bytes_per_cell": ALGO_BYTES[k], "cells_per_launch": N,
                "avg_launch_us": round(per_launch_s * 1e6, 2),
                "share": round(tot_ms / sum(v[0] for v in prof.values()), 4)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, dt, tf = cpu_baseline(blk, args.cpu_iters)
        cpu = {"value": v, "unit": "MLUP/s", "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_iters} FP64 SIP iterations of the {args.n}^3 Poisson block "
                         f"({dt:.1f} s, plain C, 1 thread)", "host": host_cpu(),
               "factor_s": round(tf, 3)}
        if ttol and "f64" in ttol:
            # the oracle's seconds per iteration times the iterations the
            # device's FP64 solve needed to reach 1e-8 (not run: extrapolated)
            its = ttol["f64"]["iterations"]
            cpu["time_to_1e-8_s"] = {"value": round(dt / args.cpu_iters * its, 1), "extrapolated": True,
                                     "iterations": its}
    line = {
        "metric": METRIC, "value": round(val_r, 1), "unit": "MLUP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_r / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"poisson_{args.n}cube", "cells": N, "alpha": 0.92, "mode": "f32_refined",
                   "inner_iters": args.inner, "corrections_per_step": args.iters,
                   "stop_rule": "none: a fixed number of corrections per step (rtol 0)",
                   "tile": dict(zip(("rows_per_thread", "tile_k", "stages"), plan_r.shape()),
                                source="measuring autotuner (sip_options.autotune), at plan creation"),
                   "parallelism": f"replicas x{world}", "l2": "working set > L2 (plan arrays "
                   f"{plan_r.nbytes() / 1e9:.2f} GB)", "step": "sip_solve on the factored plan, x reset to 0"},
        "roofline": roofline(prof_r),
        "cpu_baseline": cpu,
        "paper_cpu_context": PAPER_CPU,
        "e2e": {"value": round(val_e2e, 1), "unit": "MLUP/s", "h2d_bytes_per_step": 2 * N * 8,
                "d2h_bytes_per_step": N * 8},
        "gpu_launches": int(launches_r),
        "clocks": clk,
        "fp64": {"value": round(val_d, 1), "unit": "MLUP/s", "ms_per_step": round(ms_d / args.steps, 3),
                 "gpu_launches": int(launches_d), "roofline": roofline(prof_d),
                 "tile": dict(zip(("rows_per_thread", "tile_k", "stages"), plan_d.shape()))},
        "factor_ms": {"f32_refined": round(factor_ms_r, 2), "f64": round(factor_ms_d, 2)},
        "kernel_ms": {k: round(v[0] / max(v[1], 1), 4) for k, v in prof_r.items()},
        "kernel_ms_fp64": {k: round(v[0] / max(v[1], 1), 4) for k, v in prof_d.items()},
    }
    if ttol:
        line["time_to_1e-8"] = ttol
    if not args.no_small and world == 1:
        line["small"] = small(args, local)
    if not args.no_batched and world == 1:
        line["batched"] = batched(args, local)
    if not args.no_large and world == 1:
        line["large"] = large(args, local)
    if not args.no_assembly and world == 1:
        line["assembly"] = assembly(args, local)
    if args.serve_requests > 0 and world == 1:
        line["serving"] = serving(args, local)
    print(json.dumps(line), flush=True)
    plan_r.close()
    plan_d.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()


def tuned_options(ctx, descs, ifaces=None, **kw):
    """Options carrying the tile shape that the library's measuring autotuner
    picks for these blocks (one throw-away tuned plan, built outside every
    timed region), so that plans built from them time their factorisation
    alone."""
    from paper_1303_4538_gb300 import sip
    o = sip.default_options(autotune=1, **kw)
    p = sip.Plan(ctx, descs, o, ifaces=ifaces) if ifaces else sip.Plan(ctx, descs, o)
    q, tk, r = p.shape()
    p.close()
    return sip.default_options(rows_per_thread=q, tile_k=tk, stages=r, **kw)


def _solve_timed(plan, x, stream, rtol, max_iters, reps=1):
    """Solve from x = 0, timed with CUDA events on the plan's stream (median
    of reps); returns (ms, iterations, relres, converged)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    for _ in range(reps):
        x.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        it, rel, conv = plan.solve(rtol, max_iters)
        e1.record(stream)
        torch.cuda.synchronize()
        out.append((e0.elapsed_time(e1), it, rel, conv))
    out.sort(key=lambda r: r[0])
    return out[len(out) // 2]


def small(args, local):
    """The 32^3 convection-diffusion block (time term 0.01): latency of one
    solve to 1e-8 on a factored plan (x from 0, CUDA graphs), plain FP64 vs
    FP32-refined: p50/p99 of the host-observed call over --small-solves
    solves, and the device time (CUDA events, median of 5)."""
    import torch

    from paper_1303_4538_gb300 import sip
    from paper_1303_4538_gb300 import workloads as W

    blk = W.convdiff_32cube()
    stream = torch.cuda.current_stream()
    ctx = sip.Context(local, stream.cuda_stream)
    A = [torch.from_numpy(c).cuda() for c in blk.coef_list()]
    b = torch.from_numpy(blk.b).cuda()
    x = torch.zeros(blk.n, dtype=torch.float64, device="cuda")
    desc = sip.make_desc(blk.nx, blk.ny, blk.nz, A, b, x)
    out = {"workload": "convdiff_32cube", "cells": blk.n, "alpha": 0.92, "rtol": 1e-8, "solves": args.small_solves,
           "f32_refined_inner_iters": 4}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, mode in (("f64", sip.SIP_MODE_F64), ("f32_refined", sip.SIP_MODE_F32_REFINED)):
        plan = sip.Plan(ctx, [desc], sip.default_options(mode=mode, graphs=1))
        _solve_timed(plan, x, stream, 1e-8, 1000)
        lat = []
        for _ in range(args.small_solves):
            # one solve as a caller sees it: x reset, solve (returns on the host), result read
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x.zero_()
            it, rel, conv = plan.solve(1e-8, 1000)
            lat.append((time.perf_counter() - t0) * 1e3)
        ms_dev, _, _, _ = _solve_timed(plan, x, stream, 1e-8, 1000, reps=5)
        lat.sort()
        out[name] = {"p50_ms": round(lat[len(lat) // 2], 3), "p99_ms": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 3),
                     "device_ms": round(ms_dev, 3), "iterations": it, "relres": rel, "converged": bool(conv),
                     "MLUP_per_s": round(blk.n * it * (4 if mode == sip.SIP_MODE_F32_REFINED else 1) / ms_dev / 1e3, 1)}
        plan.close()
    ctx.close()
    return out


def large(args, local):
    """The 384^3 convection-diffusion block with median cell Peclet 10,
    coefficients stored in FP32 (factors FP32, residual and refinement FP64):
    time to 1e-8 of the refined solver at alpha 0.5 against plain FP64 SIP
    (FP64 coefficients) at alpha 0.5, and the first 40 FP64 iterations at
    alpha 0.92 (relres history: SIP diverges there)."""
    import torch

    from paper_1303_4538_gb300 import sip
    from paper_1303_4538_gb300 import workloads as W

    blk = W.convdiff_pe10_384cube()
    stream = torch.cuda.current_stream()
    ctx = sip.Context(local, stream.cuda_stream)
    A = [torch.from_numpy(c).to("cuda", torch.float32) for c in blk.coef_list()]
    b = torch.from_numpy(blk.b).cuda()
    x = torch.zeros(blk.n, dtype=torch.float64, device="cuda")
    desc = sip.make_desc(blk.nx, blk.ny, blk.nz, A, b, x, coef_dtype=1)
    out = {"workload": "convdiff_pe10_384cube", "cells": blk.n, "coefficients": "f32"}
    plan = sip.Plan(ctx, [desc], tuned_options(ctx, [desc], mode=sip.SIP_MODE_F32_REFINED, alpha=0.5, graphs=1))
    ms, it, rel, conv = _solve_timed(plan, x, stream, 1e-8, 3000)
    import numpy as np
    xs = x.cpu().numpy()
    # FP64 relative residual of the returned x under the stored FP32 matrix (widened)
    rn32, bn = ctx.residual_norm(desc)
    out["f32_refined_alpha05"] = {"seconds": round(ms / 1e3, 3), "corrections": it, "sip_iterations": it * 4,
                                  "relres": rel, "converged": bool(conv),
                                  "relres_fp64_A32": rn32 / bn,
                                  "err_vs_xstar": float(np.linalg.norm(xs - blk.xstar) / np.linalg.norm(blk.xstar))}
    plan.close()
    x_ref = x.clone()
    del A
    torch.cuda.empty_cache()
    A = [torch.from_numpy(c).cuda() for c in blk.coef_list()]
    # ... and under the FP64 matrix the generator drew
    rn64, bn64 = ctx.residual_norm(sip.make_desc(blk.nx, blk.ny, blk.nz, A, b, x_ref))
    out["f32_refined_alpha05"]["relres_fp64_A64"] = rn64 / bn64
    del x_ref
    desc = sip.make_desc(blk.nx, blk.ny, blk.nz, A, b, x)
    opt64 = tuned_options(ctx, [desc], mode=sip.SIP_MODE_F64, alpha=0.5, graphs=1)
    plan = sip.Plan(ctx, [desc], opt64)
    ms, it, rel, conv = _solve_timed(plan, x, stream, 1e-8, 5000)
    xs = x.cpu().numpy()
    out["f64_alpha05"] = {"seconds": round(ms / 1e3, 3), "iterations": it, "relres": rel, "converged": bool(conv),
                          "coefficients": "f64",
                          "err_vs_xstar": float(np.linalg.norm(xs - blk.xstar) / np.linalg.norm(blk.xstar))}
    plan.close()
    opt64.alpha = 0.92
    plan = sip.Plan(ctx, [desc], opt64)
    x.zero_()
    plan.iterate(40)
    h = plan.history()
    out["f64_alpha092_relres"] = {"min": min(h), "at_40": h[-1], "diverges": bool(h[-1] > 4 * min(h))}
    plan.close()
    ctx.close()
    if not args.no_cpu_baseline:
        # the oracle (plain C, one thread) on the same block: its factorisation
        # and one FP64 SIP iteration at alpha 0.5, and its time to 1e-8
        # extrapolated with the device's FP64 iteration count
        import oracle
        n = blk.nx
        t0 = time.perf_counter()
        F = oracle.factor(n, n, n, blk.coefs, 0.5)
        tf = time.perf_counter() - t0
        xo = np.zeros(blk.n)
        t0 = time.perf_counter()
        oracle.iterate(n, n, n, blk.coefs, F, blk.b, xo)
        ti = time.perf_counter() - t0
        its = out["f64_alpha05"]["iterations"]
        out["cpu_oracle"] = {"kind": "oracle", "cores": 1, "host": host_cpu(), "factor_s": round(tf, 2),
                             "s_per_iteration": round(ti, 3), "MLUP_per_s": round(blk.n / ti / 1e6, 1),
                             "time_to_1e-8_s": {"value": round(ti * its, 1), "extrapolated": True,
                                                "iterations": its}}
    return out


def batched(args, local):
    """The 64-block block-structured mesh (~20 M cells, sizes 24..128 per
    axis, convection-diffusion, x-chained interfaces with device-side lagged
    halo coupling): one plan over all blocks, CUDA graphs, tile shape from the
    measuring autotuner (plan creation, outside the timed region).  MLUP/s over a fixed
    number of corrections / iterations (x reset to 0, timed with CUDA events
    on the plan's stream) and the time to the 1e-8 coupled relative residual
    for the FP32-refined and the plain FP64 solver."""
    import torch

    from paper_1303_4538_gb300 import sip
    from paper_1303_4538_gb300 import workloads as W

    mesh = W.batched_mesh()
    stream = torch.cuda.current_stream()
    ctx = sip.Context(local, stream.cuda_stream)
    keep, descs, xs = [], [], []
    for blk in mesh.blocks:
        A = [torch.from_numpy(c).cuda() for c in blk.coef_list()]
        b = torch.from_numpy(blk.b).cuda()
        x = torch.zeros(blk.n, dtype=torch.float64, device="cuda")
        descs.append(sip.make_desc(blk.nx, blk.ny, blk.nz, A, b, x, symmetric=False))
        keep.append((A, b))
        xs.append(x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": "batched_mesh_64blocks", "blocks": len(mesh.blocks), "cells": mesh.n,
           "block_edges": "24..128 per axis", "generator": "convection-diffusion, x-chained interfaces"}

    def zero():
        for x in xs:
            x.zero_()

    for name, mode, inner in (("f32_refined", sip.SIP_MODE_F32_REFINED, args.inner), ("f64", sip.SIP_MODE_F64, 1)):
        ifs = [sip.sip_interface(lo, hi, nj, nk) for lo, hi, nj, nk in mesh.ifaces]
        plan = sip.Plan(ctx, descs, sip.default_options(mode=mode, inner_iters=inner, graphs=1, autotune=1),
                        ifaces=ifs)
        zero()
        plan.iterate(2)
        zero()
        torch.cuda.synchronize()
        e0.record(stream)
        plan.iterate(args.batched_iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        zero()
        torch.cuda.synchronize()
        e0.record(stream)
        it, rel, conv = plan.solve(1e-8, 20000)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"value": round(mesh.n * args.batched_iters * inner / (ms / 1e3) / 1e6, 1), "unit": "MLUP/s",
                     "tile": dict(zip(("rows_per_thread", "tile_k", "stages"), plan.shape())),
                     "ms_per_iteration": round(ms / args.batched_iters, 3),
                     "time_to_1e-8": {"seconds": round(e0.elapsed_time(e1) / 1e3, 3), "iterations": it,
                                      "sip_iterations": it * inner, "relres": rel, "converged": bool(conv)}}
        plan.close()
    # time to 1e-8 of the refined form with fewer FP32 iterations per correction
    # (interfaces exchanged after every inner FP32 iteration)
    if not args.no_inner_sweep:
        ifs = [sip.sip_interface(lo, hi, nj, nk) for lo, hi, nj, nk in mesh.ifaces]
        for m in (1, 2):
            plan = sip.Plan(ctx, descs, sip.default_options(mode=sip.SIP_MODE_F32_REFINED, inner_iters=m, graphs=1,
                                                            autotune=1), ifaces=ifs)
            zero()
            torch.cuda.synchronize()
            e0.record(stream)
            it, rel, conv = plan.solve(1e-8, 20000)
            e1.record(stream)
            torch.cuda.synchronize()
            out[f"f32_refined_m{m}_time_to_1e-8"] = {"seconds": round(e0.elapsed_time(e1) / 1e3, 3), "iterations": it,
                                                     "sip_iterations": it * m, "relres": rel,
                                                     "converged": bool(conv)}
            plan.close()
    ctx.close()
    return out


def assembly(args, local):
    """Device-side pressure-correction assembly (celp2-like) of an n^3 block
    (symmetric storage: AP, AE, AN, AT and b written): median kernel time
    over repeated launches (CUDA events on the context's stream; the working
    set of ~1.3 GB exceeds L2), its HBM roofline fraction, and the factor +
    20 FP64 SIP iterations of the assembled system from the device arrays."""
    import numpy as np
    import torch

    from paper_1303_4538_gb300 import sip
    from paper_1303_4538_gb300 import workloads as W

    n = args.n
    P = W.pcorr_inputs(n, n, n, seed=4546)
    stream = torch.cuda.current_stream()
    ctx = sip.Context(local, stream.cuda_stream)
    ins = [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (P.dx, P.dy, P.dz, P.rho, P.g, P.ux, P.uy, P.uz)]
    outs = [torch.empty(P.n, dtype=torch.float64, device="cuda") for _ in range(8)]
    outs[1] = outs[3] = outs[5] = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for r in range(13):
        e0.record(stream)
        ctx.assemble_pcorr(n, n, n, *ins, outs)
        e1.record(stream)
        torch.cuda.synchronize()
        if r >= 3:
            ms.append(e0.elapsed_time(e1))
    ms.sort()
    t = ms[len(ms) // 2]
    # per cell: rho, g (16 B) + the three face-velocity arrays (~24 B) read, 5 arrays (40 B) written;
    # 68 FP64 operations (adds and multiplies, each one op of the FP64 pipe)
    algo, ops = 80, 68
    hbm, src = peaks()
    ach_b = algo * P.n / (t / 1e3) / 1e9
    fp64_peak = 625.0   # G FP64 op/s: the nominal 1.25 TFLOP/s FP64 as 625 G fused multiply-adds per second
    ach_o = ops * P.n / (t / 1e3) / 1e9
    out = {"workload": f"pcorr_{n}cube", "cells": P.n, "storage": "symmetric (AP, AE, AN, AT, b)",
           "kernel_ms": round(t, 4), "gpu_launches_per_assembly": 1,
           "roofline": {"bound": "alu", "kernel": "assemble_pcorr", "achieved": round(ach_o, 1), "peak": fp64_peak,
                        "unit": "G FP64 op/s", "frac": round(ach_o / fp64_peak, 4),
                        "peak_source": "nominal (1.25 TFLOP/s FP64)", "fp64_ops_per_cell": ops,
                        "cells_per_launch": P.n},
           "hbm": {"achieved_GBs": round(ach_b, 1), "peak": hbm, "frac": round(ach_b / hbm, 4), "peak_source": src,
                   "algo_bytes_per_cell": algo}}
    # the assembled system feeds SIP directly from the device arrays
    x = torch.zeros(P.n, dtype=torch.float64, device="cuda")
    desc = sip.make_desc(n, n, n, outs[:7], outs[7], x, symmetric=True)
    torch.cuda.synchronize()
    e0.record(stream)
    plan = sip.Plan(ctx, [desc], sip.default_options(mode=sip.SIP_MODE_F64))
    e1.record(stream)
    torch.cuda.synchronize()
    out["factor_ms"] = round(e0.elapsed_time(e1), 2)
    e0.record(stream)
    rel = plan.iterate(20)
    e1.record(stream)
    torch.cuda.synchronize()
    out["sip_20_iterations"] = {"ms": round(e0.elapsed_time(e1), 2), "relres_before_last": rel}
    plan.close()
    ctx.close()
    return out


def serving(args, local):
    """The serving workload: ``--serve-requests`` solve requests, cube edge n
    uniform in [serve_min_n, serve_max_n], Poisson / convection-diffusion
    generator 50/50, rtol 1e-6 / 1e-8 50/50 (seeded list).  Each request's
    system is drawn on the device when it arrives (workloads.make_block_device:
    the make_block recipe with torch's generator), so the host never holds the
    request stream.  Three measurements:
      1. serial plain FP64 (plan + solve + release, one request at a time):
         service times measured on a stratified sample (7 edges spanning the
         range x 2 generators x 2 tolerances) and interpolated linearly in n
         within each generator / tolerance class for every request;
      2. saturation: the first ``serve_sat`` requests offered with a standing
         backlog (2 x slots queued), sustained solves/s of the server;
      3. Poisson arrivals at 0.8 x the measured saturation rate over all
         requests: per-request latency (arrival -> result seen by the host),
         p50 / p99, solves/s.  The serial FP64 queue is replayed (FIFO, the
         interpolated service times) on the same arrivals and at 0.8 x its own
         capacity;
      4. the first ``serve_capacity_prefix`` requests with Poisson arrivals at
         0.8 x the serial FP64 capacity, served and replayed serially.
    Server: FP32-refined mode, CUDA graphs, ``serve_slots`` slots, admitted
    by HBM footprint."""
    import numpy as np
    import torch

    from paper_1303_4538_gb300 import sip
    from paper_1303_4538_gb300 import workloads as W

    rng = np.random.Generator(np.random.PCG64(4543))
    N = args.serve_requests
    lo, hi = args.serve_min_n, args.serve_max_n
    reqs = [(int(rng.integers(lo, hi + 1)), "poisson" if rng.random() < 0.5 else "convdiff",
             1e-6 if rng.random() < 0.5 else 1e-8) for _ in range(N)]
    gs = torch.cuda.Stream()
    ctx = sip.Context(local, gs.cuda_stream)

    def draw(n, kind, seed):
        with torch.cuda.stream(gs):
            c, b, _ = W.make_block_device(n, n, n, seed, kind)
            x = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
        gs.synchronize()
        coefs = list(c)
        if kind == "poisson":
            coefs[1] = coefs[3] = coefs[5] = None
        return sip.make_desc(n, n, n, coefs, b, x, symmetric=(kind == "poisson")), (c, b, x)

    # 1. serial plain FP64 on a stratified sample
    o64 = sip.default_options(mode=sip.SIP_MODE_F64)
    edges = sorted(set(int(round(v)) for v in np.linspace(lo, hi, 7)))
    d, keep = draw(lo, "convdiff", 1)
    p = sip.Plan(ctx, [d], o64)
    p.solve(1e-6, 5000)   # warm-up (module load, pool)
    p.close()
    svc = {}
    for kind in ("poisson", "convdiff"):
        for rtol in (1e-6, 1e-8):
            ts = []
            for n in edges:
                d, keep = draw(n, kind, 7 * n + (kind == "poisson"))
                gs.synchronize()
                t0 = time.perf_counter()
                p = sip.Plan(ctx, [d], o64)
                p.solve(rtol, 50000)
                p.close()
                gs.synchronize()
                ts.append(time.perf_counter() - t0)
                del keep
            svc[(kind, rtol)] = ts
    serv = np.array([float(np.interp(n, edges, svc[(kind, rtol)])) for n, kind, rtol in reqs])
    cap_ser = 1.0 / float(serv.mean())

    oref = sip.default_options(mode=sip.SIP_MODE_F32_REFINED, graphs=1)
    slots = args.serve_slots

    def run(count, arrivals):
        """Serve requests 0..count-1; arrivals None: a standing backlog of
        2 x slots; else arrival times (s).  Returns (latencies, finish times, t0, failed, stats)."""
        srv = sip.Server(ctx, 200 << 30, slots)
        lat, fin = np.zeros(count), np.zeros(count)
        pending, bad = {}, 0
        i = done = 0
        t0 = time.perf_counter()
        arr = np.zeros(count) if arrivals is None else arrivals
        while done < count:
            now = time.perf_counter() - t0
            while i < count and ((arrivals is None and len(pending) < 2 * slots) or
                                 (arrivals is not None and arr[i] <= now)):
                n, kind, rtol = reqs[i]
                d, keep = draw(n, kind, 4543 * 1000 + i)
                if arrivals is None:
                    arr[i] = time.perf_counter() - t0
                pending[srv.submit(d, oref, rtol, 50000, keep=keep)] = i
                i += 1
                now = time.perf_counter() - t0
            for t in list(pending):
                res = srv.poll(t)
                if res is not None:
                    k = pending.pop(t)
                    fin[k] = time.perf_counter() - t0
                    lat[k] = fin[k] - arr[k]
                    bad += res[0] != sip.SIP_OK
                    done += 1
            time.sleep(0.0002)
        st = srv.stats()
        srv.stop()
        return lat, fin, arr, bad, st

    # 2. saturation on a prefix
    nsat = min(args.serve_sat, N)
    lat_s, fin_s, arr_s, bad_s, st_s = run(nsat, None)
    mu = nsat / float(fin_s.max())
    # 3. Poisson arrivals at 0.8 x the saturation rate
    lam = 0.8 * mu
    arr = np.cumsum(np.random.Generator(np.random.PCG64(4548)).exponential(1.0 / lam, size=N))
    lat, fin, arr, bad, st = run(N, arr)
    # 4. a prefix of the list with arrivals at 0.8 x the serial FP64 capacity
    #    (all 2000 at that rate would take ~20 minutes of arrivals)
    npre = min(args.serve_capacity_prefix, N)
    pre = None
    if npre > 0:
        arr_p = np.cumsum(np.random.Generator(np.random.PCG64(4550)).exponential(1.0 / (0.8 * cap_ser), size=npre))
        lat_p, fin_p, arr_p, bad_p, _ = run(npre, arr_p)
        end, lat_sp = 0.0, []
        for a_, s_ in zip(arr_p, serv[:npre]):
            end = max(a_, end) + s_
            lat_sp.append(end - a_)
        pre = (npre, arr_p, lat_p, fin_p, bad_p, np.array(lat_sp))
    ctx.close()

    def replay(arrivals):
        end, out = 0.0, []
        for a, s_ in zip(arrivals, serv):
            end = max(a, end) + s_
            out.append(end - a)
        return np.array(out)

    ms = lambda v, q: round(float(np.percentile(np.asarray(v) * 1e3, q)), 1)
    arr_ser = np.cumsum(np.random.Generator(np.random.PCG64(4549)).exponential(1.0 / (0.8 * cap_ser), size=N))
    lat_same, lat_own = replay(arr), replay(arr_ser)
    return {"requests": N, "sizes": f"cubes {lo}..{hi} (edge uniform)", "mix": "Poisson/conv-diff 50/50, rtol 1e-6/1e-8",
            "inputs": "drawn on the device at arrival (make_block recipe, torch generator)",
            "served": {"mode": "f32_refined (4 FP32 iterations per correction), CUDA graphs", "slots": slots,
                       "saturation": {"requests": nsat, "solves_per_s": round(mu, 2), "seconds": round(float(fin_s.max()), 1),
                                      "failed": int(bad_s)},
                       "poisson_arrivals": {"arrivals_per_s": round(lam, 2), "load": "0.8 x saturation",
                                            "solves_per_s": round(N / float(fin.max() - arr[0]), 2),
                                            "wall_s": round(float(fin.max()), 1),
                                            "p50_ms": ms(lat, 50), "p99_ms": ms(lat, 99), "failed": int(bad),
                                            "peak_admitted_bytes": int(st["peak_in_use_bytes"]),
                                            "slot_busy_s": round(st["busy_ms"] / 1e3, 1)}},
            "serial_fp64": {"capacity_solves_per_s": round(cap_ser, 3),
                            "service_time_sample": {"edges": edges, "classes": "poisson/convdiff x 1e-6/1e-8",
                                                    "seconds": {f"{k}_{r:g}": [round(v, 3) for v in t]
                                                                for (k, r), t in svc.items()}},
                            "replay_same_arrivals": {"p50_ms": ms(lat_same, 50), "p99_ms": ms(lat_same, 99)},
                            "replay_at_0.8_own_capacity": {"arrivals_per_s": round(0.8 * cap_ser, 3),
                                                           "p50_ms": ms(lat_own, 50), "p99_ms": ms(lat_own, 99)}},
            "vs_serial_fp64_capacity": round(mu / cap_ser, 2),
            "at_0.8_serial_capacity": None if pre is None else {
                "requests": pre[0], "note": "the first requests of the list; arrivals at 0.8 x the serial FP64 capacity",
                "arrivals_per_s": round(0.8 * cap_ser, 3),
                "served": {"p50_ms": ms(pre[2], 50), "p99_ms": ms(pre[2], 99), "failed": int(pre[4]),
                           "solves_per_s": round(pre[0] / float(pre[3].max() - pre[1][0]), 3)},
                "serial_fp64_replay": {"p50_ms": ms(pre[5], 50), "p99_ms": ms(pre[5], 99)}}}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
