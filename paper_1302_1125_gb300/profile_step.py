"""Run a few fused steps of one workload, for kernel profiling.

    python -m paper_1302_1125_gb300.profile_step --workload cloud_3d --scale 2 \
        --precision fp32 --steps 3 --warmup 2

Initialises the workload on the GPU, runs `warmup` steps, then `steps`
steps, and prints the CUDA-event time per step.  The grid shrinks by
`scale` per axis so that a profiler capture stays small.
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
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cloud_3d", choices=sorted(MAKERS))
    ap.add_argument("--scale", type=int, default=1)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    a = ap.parse_args()
    B.build()
    w = MAKERS[a.workload](a.scale)
    prec = rlb.FP32_STORAGE if a.precision == "fp32" else rlb.FP64
    g = rlb.Grid.from_workload(w, precision=prec)
    g.init(*[torch.as_tensor(x, device="cuda") for x in w.fields()])
    g.step(a.warmup)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    g.step(a.steps)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / max(a.steps, 1)
    print(json.dumps({"workload": w.name, "cells": w.N, "precision": a.precision,
                      "ms_per_step": ms, "mlups": w.N / (ms * 1e-3) / 1e6}))


if __name__ == "__main__":
    main()
