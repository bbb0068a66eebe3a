"""Run a few steps of one workload through the library, for profiler
captures (ncu) of individual kernels on cases larger than L2.

  python -m paper_2111_11806_gb300.profile_case --workload cylinder --n 4096 --precision fp32 --steps 3

Prints the per-kernel CUDA-event times of the steps it ran.
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cylinder", choices=["cylinder", "dynamic", "impact", "sphere"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--batch", type=int, default=0, help="run a batch of this many ellipse instances instead")
    args = ap.parse_args(argv)
    if args.batch:
        return run_batch(args)
    import torch
    import workloads as W
    from paper_2111_11806_gb300 import binding as B
    B.load()
    make = {"cylinder": lambda n: W.cylinder_2d(n), "dynamic": lambda n: W.dynamic_body_2d(n, n // 2),
            "impact": lambda n: W.impact_2d(n), "sphere": lambda n: W.sphere_3d(n)}[args.workload]
    wl = make(args.n)
    prec = B.DFV_FP32 if args.precision == "fp32" else B.DFV_FP64
    stream = torch.cuda.Stream()
    g = B.Grid.from_workload(wl, precision=prec, stream=stream)
    g.run(1, wl.cfl)
    g.profile(True)
    for _ in range(args.steps):
        g.run(1, wl.cfl, sync=False)
    ms, n = g.profile(False)
    g.check(timeout_ms=120000)
    print(json.dumps({"workload": wl.name, "precision": args.precision, "cells": wl.ncell, "steps": n,
                      "ms_per_step": {"seed": ms[0] / n, "stage1": ms[1] / n, "stage2": ms[2] / n,
                                      "stage3": ms[3] / n, "finalize": ms[4] / n}}))
    return 0


def run_batch(args):
    import torch
    import workloads as W
    from paper_2111_11806_gb300 import binding as B
    B.load()
    wls = [W.ellipse_instance(i) for i in range(args.batch)]
    prec = B.DFV_FP32 if args.precision == "fp32" else B.DFV_FP64
    stream = torch.cuda.Stream()
    bt = B.Batch(wls, precision=prec, stream=stream)
    bt.set_all_fields()
    # the schedule the autotuner picks for the 256-ellipse batch: one CTA
    # per four work items, largest instances first
    bt.set_schedule(0, 1)
    bt.run(1, 0.8)
    bt.profile(True)
    bt.run(args.steps, 0.8)
    ms, n = bt.profile(False)
    bt.time(0)
    print(json.dumps({"workload": "batch_%d_ellipses" % args.batch, "precision": args.precision,
                      "cells": bt.total_cells, "steps": n,
                      "ms_per_step": {"seed": ms[0] / n, "stage1": ms[1] / n, "stage2": ms[2] / n,
                                      "stage3": ms[3] / n}}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
