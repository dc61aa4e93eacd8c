"""Run a few fused steps of one workload, for kernel profiling.

    python -m paper_1302_1125_gb300.profile_step --workload cloud_3d --scale 2 \
        --precision fp32 --steps 3 --warmup 2

Initialises the workload on the GPU, runs `warmup` steps, then `steps`
steps, and prints the CUDA-event time per step.  The grid shrinks by
`scale` per axis so that a profiler capture stays small.

    python -m paper_1302_1125_gb300.profile_step --workload batch_tubes --scale 8 --steps 1 --warmup 1

runs the batched tubes instead: a sweep of 512/scale tubes drawn like the
512-tube sweep (same seed and distributions), each for 4 Nx / scale steps
per launch (`steps` launches after
`warmup` launches), with the given launch shape (--tuning threads,bound,
cluster,pairs_per_thread; default: the library's).
"""
from __future__ import annotations

import argparse
import json

import torch

from . import build as B
from . import rlb
from . import workloads as W

MAKERS = {
    "cloud_3d": lambda s: W.cloud_3d(scale=s),
    "cloud_2d": lambda s: W.cloud_2d(scale=s),
    "tube_8192a": lambda s: W.tube_8192("a", nx=8192 // s),
    "tube_800": lambda s: W.tube_800(),
    "batch_tubes": None,
}


def run_batch(a):
    import numpy as np
    full = W.batch_tubes()
    k = max(1, full.B // a.scale)
    spec = W.batch_tubes(count=k)
    steps = np.maximum(spec.steps // a.scale, 1)
    b = rlb.Batch.from_spec(spec, symmetry_1d=int(a.symmetry))
    if a.tuning:
        b.set_tuning(*[int(v) for v in a.tuning.split(",")])
    b.init(*spec.fields())
    for _ in range(a.warmup):
        b.step(steps)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for _ in range(a.steps):
        b.step(steps)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / max(a.steps, 1)
    upd = float(np.sum(spec.nx.astype(np.float64) * steps))
    t, ncl = b.tuning()
    print(json.dumps({"workload": f"batch_tubes(count={k}), steps 4 Nx / {a.scale}", "tubes": k,
                      "cell_updates": upd, "ms_per_launch": ms, "mlups": upd / (ms * 1e-3) / 1e6,
                      "tuning": t.as_dict(), "resident_clusters": ncl}))


def arg_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cloud_3d", choices=sorted(MAKERS))
    ap.add_argument("--scale", type=int, default=1)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_rec64", "fp64"],
                    help="fp32_rec64: FP32 storage with the FP64 recovery (recovery_fp64 = 1)")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--mapping", type=int, default=0,
                    help="grids: rlb_options.thread_mapping (0 automatic, 1 tiles, 2 linear, 3 tiles staged by block-wide bulk copies)")
    ap.add_argument("--tuning", default="", help="batch launch shape threads,bound,cluster,pairs_per_thread")
    ap.add_argument("--symmetry", action="store_true", help="batch: the 1-D symmetry reduction")
    return ap


def main():
    a = arg_parser().parse_args()
    B.build()
    if a.workload == "batch_tubes":
        return run_batch(a)
    w = MAKERS[a.workload](a.scale)
    prec = rlb.FP64 if a.precision == "fp64" else rlb.FP32_STORAGE
    g = rlb.Grid.from_workload(w, precision=prec, recovery_fp64=int(a.precision == "fp32_rec64"),
                               thread_mapping=a.mapping)
    g.init(*[torch.as_tensor(x, device="cuda") for x in w.fields()])
    g.step(a.warmup)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    g.step(a.steps)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / max(a.steps, 1)
    print(json.dumps({"workload": w.name, "cells": w.N, "precision": a.precision, "kernel": g.step_kernel,
                      "ms_per_step": ms, "mlups": w.N / (ms * 1e-3) / 1e6}))


if __name__ == "__main__":
    main()
