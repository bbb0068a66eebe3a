#!/usr/bin/env python
"""Benchmark of the diffuse rigid-body finite-volume update (arXiv:2111.11806)
on GB300: cell-updates/s of the FP32 bulk form against the plain FP64 form,
with the HBM roofline fraction of the dominant kernel (the SSP-RK3 stage).

Workload: 2-D Mach 3 shock over a static rigid cylinder, 512 x 512 cells, air,
CFL 0.8 (the metric's quoted configuration).  One benchmark step = one solver
time step (seeding, three RK stages, CFL and force reductions).  The state
(5.2 MB in FP32) fits in L2, so L2 is flushed (a 256 MiB write) before every
timed step and only the step itself is inside its CUDA-event window.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on the same
workload (each benchmark step: one oracle time step on a bounded sample of
the grid's rows).  Under torchrun every rank runs an independent replica
(the single-grid workload does not shard); the whole-job value sums the
replicas' cell updates over the slowest rank's time.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s FP32 & batched vs plain FP64 at stated L1 error; % HBM roofline"
UNIT = "cell-updates/s"
WORKLOAD = "cylinder_2d_512x512_mach3_cfl0.8"
N_CELL = 512 * 512
KERNEL_SOURCES = ["paper_2111_11806_gb300/csrc/dfv_device.cuh", "paper_2111_11806_gb300/csrc/dfv_kernels.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-count", type=int, default=256)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per stage launch from the committed ncu summary, if the
    kernel sources still match the ones it was captured from."""
    p = os.path.join(ROOT, "profiles", "rk_stage_cylinder_512_fp32.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_source_hash") != kernel_hash():
        return None
    return d.get("dram_bytes_per_stage_launch")


class Clocks:
    """nvidia-smi sampler running while the timed work runs."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-i", str(index), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(max_seconds, rows=None):
    """FP64 oracle cell-updates/s on the benchmark workload (one core)."""
    import numpy as np
    import workloads as W
    from oracle import Oracle
    wl = W.cylinder_2d(512)
    if rows is not None and rows < 512:
        # bounded sample: the band of `rows` rows through the body's centre
        lo_row = 256 - rows // 2
        prim = wl.prim.reshape(wl.nvar, 512, 512)[:, lo_row:lo_row + rows, :].reshape(wl.nvar, -1)
        o = Oracle(2, (512, rows), (0.0, lo_row / 512.0), (1.0, (lo_row + rows) / 512.0), wl.materials)
        o.set_prim(np.ascontiguousarray(prim))
        cells = 512 * rows
    else:
        o = Oracle.from_workload(wl)
        cells = N_CELL
    steps, t0 = 0, time.perf_counter()
    while True:
        o.step(o.compute_dt(0.8))
        steps += 1
        el = time.perf_counter() - t0
        if el >= max_seconds:
            break
    return cells * steps / el, "%d oracle steps on a 512x%d band of the 512x512 grid in %.1f s" % (
        steps, cells // 512, el)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import workloads as W
    from oracle import Oracle
    import oracle
    oracle.build()
    wl = W.cylinder_2d(512)
    # bounded sample: rows of the grid per benchmark step so that the run stays within ~2 minutes
    budget_s = 120.0
    per_step_full = 0.6
    frac = min(1.0, budget_s / max(1.0, (args.steps + args.warmup) * per_step_full))
    rows = max(8, int(512 * frac) // 8 * 8)
    lo_row = 256 - rows // 2
    prim = wl.prim.reshape(wl.nvar, 512, 512)[:, lo_row:lo_row + rows, :].reshape(wl.nvar, -1)
    o = Oracle(2, (512, rows), (0.0, lo_row / 512.0), (1.0, (lo_row + rows) / 512.0), wl.materials)
    o.set_prim(np.ascontiguousarray(prim))
    for _ in range(args.warmup):
        o.step(o.compute_dt(0.8))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(o.compute_dt(0.8))
    el = time.perf_counter() - t0
    cells = 512 * rows
    value = cells * args.steps / el
    sample = "each step: one FP64 oracle step on the 512x%d band through the body of the 512x512 grid" % rows
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "global_batch": 1, "cells": cells, "precision": "fp64",
                       "l2": "host run"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_steps(torch, g, stream, flush, steps, profile):
    """Per-step CUDA-event windows with an L2 flush before each step."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if profile:
        g.profile(True)
    n0 = g.launch_count()
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(k & 0x7F)
            starts[k].record(stream)
            g.run(1, 0.8, sync=False)
            ends[k].record(stream)
    stream.synchronize()
    launches = g.launch_count() - n0
    prof = g.profile(False) if profile else None
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return ms, launches, prof


def run_batched(torch, B, W, stream, args):
    """Batched workload: per-step CUDA-event timing of graph replays, per-phase
    profile for the stage-kernel roofline, and the plain FP64 batch."""
    peak, peak_kind = measured_peaks()
    wls = [W.ellipse_instance(i) for i in range(args.batch_count)]
    cells = int(sum(int(np.prod(wl.n)) for wl in wls))
    out = {"workload": "ellipses_%d_instances_128-512sq_fp32" % args.batch_count, "cells": cells}
    for prec, key in ((B.DFV_FP32, "fp32"), (B.DFV_FP64, "fp64")):
        bt = B.Batch(wls, precision=prec, stream=stream)
        bt.set_all_fields()
        choice = bt.autotune(trial_steps=2, cfl=0.8)
        bt.run(3, 0.8)
        k = 30 if prec == B.DFV_FP32 else 4
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = bt.launch_count()
        stream.synchronize()
        e0.record(stream)
        bt.run(k, 0.8)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        launches = bt.launch_count() - n0
        bt.profile(True)
        bt.run(3, 0.8)
        pms, pn = bt.profile(False)
        w = 4 if prec == B.DFV_FP32 else 8
        nvar = bt.nvar
        stage_ms = float(pms[1] + pms[2] + pms[3]) / pn
        achieved = 8 * nvar * w * cells / (stage_ms * 1e-3) / 1e9
        rec = {"value": cells * k / (ms * 1e-3), "unit": UNIT, "steps": k, "ms_per_step": ms / k,
               "autotune": {"ctas_per_sm": choice[0] if choice[0] > 0 else "one CTA per work item",
                            "schedule": ["instance-order static", "largest-first static",
                                         "largest-first dynamic"][choice[1]]},
               "gpu_launches": int(launches),
               "phase_ms_per_step": {"seed": pms[0] / pn, "stage1": pms[1] / pn, "stage2": pms[2] / pn,
                                     "stage3": pms[3] / pn},
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "peak_kind": peak_kind,
                            "kernel": "k_batch_stage (3 launches per step)",
                            "algorithmic_bytes_per_step": 8 * nvar * w * cells}}
        out[key] = rec
        del bt
        torch.cuda.synchronize()
    out["fp32_over_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    return out


def run_sphere(torch, B, W, stream):
    """256^3 sphere workload, FP32: event-timed steps and the stage roofline."""
    peak, peak_kind = measured_peaks()
    wl = W.sphere_3d(256)
    g = B.Grid.from_workload(wl, precision=B.DFV_FP32, stream=stream)
    g.run(2, 0.8)
    k = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    g.run(k, 0.8)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    g.profile(True)
    g.run(3, 0.8)
    pms, pn = g.profile(False)
    stage_ms = float(pms[1] + pms[2] + pms[3]) / pn
    achieved = 8 * wl.nvar * 4 * wl.ncell / (stage_ms * 1e-3) / 1e9
    del g
    return {"workload": "sphere_3d_256^3_mach2.5_fp32", "cells": wl.ncell, "value": wl.ncell * k / (ms * 1e-3),
            "unit": UNIT, "steps": k, "ms_per_step": ms / k,
            "phase_ms_per_step": {"seed": pms[0] / pn, "stage1": pms[1] / pn, "stage2": pms[2] / pn,
                                  "stage3": pms[3] / pn},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "kernel": "k_stage_z (3-D FP32, marching along z)"}}


def run_ours(args):
    rank, world, local = dist_env()
    import numpy as np
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import workloads as W
    from paper_2111_11806_gb300 import binding as B
    B.load()

    wl = W.cylinder_2d(512)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    g32 = B.Grid.from_workload(wl, precision=B.DFV_FP32, device=dev, stream=stream)
    g64 = B.Grid.from_workload(wl, precision=B.DFV_FP64, device=dev, stream=stream)

    clocks = Clocks(local) if rank == 0 else None
    # warm-up (untimed)
    g32.run(args.warmup, 0.8)
    g64.run(max(3, args.warmup // 2), 0.8)
    torch.cuda.synchronize()

    # --- kernel-only timed region: FP32 form (the headline)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # one graph replay per step, no per-kernel events inside the step
    ms32, launches32, _ = time_steps(torch, g32, stream, flush, args.steps, profile=False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # second timed pass of the same workload with CUDA events around every
    # kernel (launched one by one) for the per-kernel durations of the roofline
    kprof = max(20, min(args.steps, 200))
    msp32, _, prof32 = time_steps(torch, g32, stream, flush, kprof, profile=True)
    total_ms = sum(ms32)
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    value = world * args.steps * N_CELL / (total_ms * 1e-3)

    # --- plain FP64 form, same procedure, fewer steps
    k64 = max(5, min(args.steps, 50))
    ms64, launches64, _ = time_steps(torch, g64, stream, flush, k64, profile=False)
    value64 = world * k64 * N_CELL / (sum(ms64) * 1e-3)

    # --- end to end through the C ABI with host buffers: fields in from pinned
    # host memory, the configuration's 500 steps, fields back to the host
    job_steps = wl.steps
    nvar = wl.nvar
    host_in = torch.empty((nvar, N_CELL), dtype=torch.float64, pin_memory=True)
    host_in.numpy()[:] = wl.prim
    host_out = torch.empty((nvar, N_CELL), dtype=torch.float64, pin_memory=True)
    g_e2e = B.Grid(wl.dim, wl.n, wl.lo, wl.hi, wl.materials, precision=B.DFV_FP32, device=dev, stream=stream)
    jobs = 2
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(jobs):
        g_e2e.set_fields(host_in.numpy())
        g_e2e.set_body()
        g_e2e.run(job_steps, 0.8)
        g_e2e.get_fields(B.DFV_FIELDS_PRIMITIVE, out=host_out.numpy())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = world * jobs * job_steps * N_CELL / e2e_s
    bytes_io = nvar * N_CELL * 8

    # --- batched form: 256 independent instances of {128..512}^2 (about 27 M
    # cells, 0.54 GB per FP32 state copy: larger than L2, so no flush is needed),
    # persistent launches over the (instance, tile) work list in a CUDA graph,
    # schedule chosen by the autotuner
    batched = None
    if not args.no_batched:
        batched = run_batched(torch, B, W, stream, args)

    # --- 3-D: Mach 2.5 shock over a rigid sphere, 256^3 cells (0.40 GB per FP32 state copy)
    sphere = None
    if not args.no_batched:
        sphere = run_sphere(torch, B, W, stream)

    clk = clocks.stop() if clocks else None

    # --- accuracy of the FP32 form after the timed steps: relative L1 of the
    # density against the FP64 form advanced the same number of steps
    warm32 = args.warmup + args.steps
    g_acc32 = B.Grid.from_workload(wl, precision=B.DFV_FP32, device=dev, stream=stream)
    g_acc64 = B.Grid.from_workload(wl, precision=B.DFV_FP64, device=dev, stream=stream)
    nacc = 200
    g_acc32.run(nacc, 0.8)
    g_acc64.run(nacc, 0.8)
    r32, r64 = g_acc32.prim()[0], g_acc64.prim()[0]
    l1 = float(np.abs(r32 - r64).sum() / np.abs(r64).sum())
    row = lambda r: np.argmax(np.abs(np.diff(r.reshape(512, 512)[256])))
    shock_cells = int(abs(row(r32) - row(r64)))

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    peak, peak_kind = measured_peaks()
    w32 = 4
    stage_ms = float(prof32[0][1] + prof32[0][2] + prof32[0][3])
    stage_launches = 3 * prof32[1]
    bytes_per_launch = 8 * nvar * w32 * N_CELL / 3.0    # (2 + 3 + 3) nvar planes over the 3 stage launches
    achieved = bytes_per_launch / (stage_ms * 1e-3 / stage_launches) / 1e9
    traffic = recorded_traffic()
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, sample = oracle_rate(15.0, rows=128)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": world, "cells_per_gpu": N_CELL, "nvar": nvar,
                   "precision": "fp32 bulk (FP64 polar/closure where phi<1e-6)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed (256 MiB write) before every timed step"},
        "fp64": {"value": value64, "unit": UNIT, "steps": k64, "ms_per_step": sum(ms64) / k64,
                 "fp32_over_fp64": value / value64},
        "accuracy": {"fp32_vs_fp64_rel_l1_density": l1, "shock_position_diff_cells": shock_cells,
                     "after_steps": nacc},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "k_stage (SSP-RK3 stage), FP32",
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "avg_launch_ms": stage_ms / stage_launches,
                     "timing": "CUDA events around each kernel in a second timed pass of %d steps "
                               "(launched one by one; that pass took %.4f ms per step)" % (kprof, sum(msp32) / kprof)},
        "kernel_ms_per_step": {"seed": prof32[0][0] / prof32[1], "stage1": prof32[0][1] / prof32[1],
                               "stage2": prof32[0][2] / prof32[1], "stage3": prof32[0][3] / prof32[1],
                               "finalize": prof32[0][4] / prof32[1]},
        "cpu_baseline": cpu,
        "batched": batched,
        "sphere_3d": sphere,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": bytes_io / job_steps,
                "d2h_bytes_per_step": bytes_io / job_steps,
                "job": "set_fields(host) + %d steps + get_fields(host), %d jobs" % (job_steps, jobs)},
        "gpu_launches": int(launches32),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
