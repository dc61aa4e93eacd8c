#!/usr/bin/env python
"""Throughput of the fused RLB time step on GB300.

Workload: the 3-D shock-cloud, 512 x 256 x 256 cells (33.5 M), FP32
population storage and arithmetic (moment sums in double-float, i.e. float
pairs; no FP64 instruction); a step is one time step
of the whole grid (every cell: minmod streaming of 38 populations, bulk
Laplacian, moments, Landau recovery, equilibria, implicit update).  The FP64
form is timed on the same grid for the FP32/FP64 ratio, and the FP32 form's
L1 error against the FP64 form is measured on the 800-cell tube.  The
512-tube batched sweep (one persistent launch) is reported under "batch",
next to a sample of the same tubes run one by one.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas (the step has no exchange
between ranks in this configuration); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM peak; FP32-storage vs FP64 form at stated L1 error"
UNIT = "MLUPS"
# algorithmic bytes per cell update: 38 populations read and written once,
# 5 previous-level macroscopic values read and written once
BYTES_FP32 = 38 * 4 * 2 + 5 * 4 * 2     # 344
BYTES_FP64 = 38 * 8 * 2 + 5 * 8 * 2     # 688
# 1-D symmetry reduction: 14 class planes and 3 previous-level planes
BYTES_SYM1D = 14 * 4 * 2 + 3 * 4 * 2    # 136
# 2-D symmetry reduction: 14 f + 14 h class planes, 4 previous-level planes
BYTES_SYM2D = 28 * 4 * 2 + 4 * 4 * 2    # 256


def csrc_hash(files=None) -> str:
    """sha256 (first 16 hex) of the named kernel sources (all of csrc/ if None)"""
    import hashlib
    d = os.path.join(ROOT, "paper_1302_1125_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(files if files else os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(summary: str, units: float):
    """DRAM bytes per launch from the committed ncu summary of a kernel (bytes
    per unit x units), or None if that kernel's sources changed since the
    capture"""
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
    except OSError:
        return None
    keys = ("csrc_sha256:", "csrc_files:", "traffic_bytes_per_cell:")
    fields = dict(ln.split(":", 1) for ln in text.splitlines() if ln.startswith(keys))
    files = fields.get("csrc_files", "").split() or None
    if fields.get("csrc_sha256", "").split()[0:1] != [csrc_hash(files)]:
        return None
    return float(fields["traffic_bytes_per_cell"].split()[0]) * units


def profiled_value(summary: str, key: str):
    """a per-unit figure (first number after `key:`) from a committed ncu
    summary, or None if the kernel's sources changed since the capture"""
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
    except OSError:
        return None
    keys = ("csrc_sha256:", "csrc_files:", key + ":")
    fields = dict(ln.split(":", 1) for ln in text.splitlines() if ln.startswith(keys))
    files = fields.get("csrc_files", "").split() or None
    if key not in fields or fields.get("csrc_sha256", "").split()[0:1] != [csrc_hash(files)]:
        return None
    return float(fields[key].split()[0])


# GB300: 152 SMs, 4 warp schedulers each issuing one warp instruction per
# clock, and an FP64 pipe of 2 lanes per SM (1.26 TFLOP/s of FMA at 2.07 GHz)
N_SM = 152
SCHEDULERS_PER_SM = 4
DP_LANES_PER_SM = 2


def alu_roofline(ops_per_unit, units_per_s, lanes_per_clk, clk, what):
    """achieved / peak of an arithmetic pipe: ops per unit (from the committed
    profile) x units per second, against lanes per clock x the median SM
    clock sampled in the timed region"""
    if ops_per_unit is None or clk is None or not clk.get("sm_mhz"):
        return None
    mhz = clk["sm_mhz"]
    achieved = ops_per_unit * units_per_s / 1e9
    peak = lanes_per_clk * mhz * 1e6 / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G ops/s", "frac": achieved / peak,
            "ops_per_unit": ops_per_unit, "sm_mhz": mhz, "what": what}


def issue_roofline(instr_per_unit, units_per_s, clk, what):
    """achieved / peak warp-instruction issue: thread-instructions per unit
    (the committed profile's warp instructions x 32 / units) / 32 x units
    per second, against 4 schedulers x 152 SMs x the sampled SM clock"""
    if instr_per_unit is None or clk is None or not clk.get("sm_mhz"):
        return None
    mhz = clk["sm_mhz"]
    achieved = instr_per_unit / 32.0 * units_per_s / 1e9
    peak = N_SM * SCHEDULERS_PER_SM * mhz * 1e6 / 1e9
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "G warp-instructions/s",
            "frac": achieved / peak, "thread_instructions_per_unit": instr_per_unit, "sm_mhz": mhz,
            "what": what}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region"""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.first = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once nvidia-smi delivers samples (its
            # start-up takes longer than a short timed region)
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.first = len(self.lines)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def mark(self) -> int:
        """the number of samples so far (a boundary between regions)"""
        return len(self.lines)

    def summary(self, lo=None, hi=None):
        """median SM clock and throttle reasons of the samples [lo, hi)
        (default: from the start of the timed region); a region shorter
        than the sampling interval gets the sample taken nearest after it"""
        lo = self.first if lo is None else lo
        hi = len(self.lines) if hi is None else hi
        lines = self.lines[lo:hi] or self.lines[hi:hi + 1] or self.lines[-1:]
        if not lines:
            return None
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def rejected(clk):
    if clk is None:
        return False
    if set(clk["reasons"]) & {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}:
        return True
    return clk["sm_max_mhz"] and clk["sm_mhz"] < 0.6 * clk["sm_max_mhz"] and not clk["reasons"]


def timed_steps(torch, g, steps, warmup, device_index, window_s=0.0):
    """warm up, then time `steps` steps with CUDA events on the launching
    stream.  With window_s > 0 and a timed region shorter than that, the same
    steps are repeated afterwards for about window_s seconds (the clock
    window), timed the same way, so that the clock samples (every 50 ms)
    cover the kernel running for long enough to mean something; the window
    is reported beside the timed region, not in its place."""
    g.step(warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    window = None
    for attempt in range(2):
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(device_index) as cs:
            barrier()
            torch.cuda.synchronize()
            l0 = g.launches
            start.record(stream)
            g.step(steps)
            end.record(stream)
            torch.cuda.synchronize()
            barrier()
            mid = cs.mark()
            ms = start.elapsed_time(end)
            launches = g.launches - l0
            if window_s > 0.0 and ms < 1e3 * window_s:
                reps = max(1, int(math.ceil(1e3 * window_s / max(ms, 1e-3))))
                w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                w0.record(stream)
                for _ in range(reps):
                    g.step(steps)
                w1.record(stream)
                torch.cuda.synchronize()
                wms = w0.elapsed_time(w1)
                window = {"steps": reps * steps, "ms_per_step": wms / (reps * steps),
                          "clocks": cs.summary(mid, cs.mark())}
        clk = cs.summary(cs.first, mid)
        if not rejected(clk):
            break
    return ms, clk, launches, window


_dist = None


def barrier():
    if _dist is not None:
        _dist.barrier()


def max_over_ranks(torch, v: float) -> float:
    """the largest v over the ranks (the job's time is its slowest replica's)"""
    if _dist is None:
        return v
    dev = "cuda" if _dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    _dist.all_reduce(t, op=_dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, units_per_rank: float, seconds: float) -> float:
    """whole-job throughput in millions of units per second: every replica
    processes units_per_rank in the (max-over-ranks) time"""
    return world * units_per_rank / seconds / 1e6


def cpu_baseline(steps=None, warmup=1, budget_s=12.0):
    """the oracle, as it stands, on a bounded sample of the workload: the same
    shock-cloud shrunk 8x per axis (64 x 32 x 32 cells), FP64, all host cores"""
    import oracle
    from paper_1302_1125_gb300 import workloads as W
    oracle.set_threads(os.cpu_count() or 1)
    w = W.cloud_3d(scale=8, precision=W.FP64)
    p = oracle.Params(nx=w.nx, ny=w.ny, nz=w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, dt=w.dt_over_dx,
                      eta_over_s=w.eta_over_s, zeta_over_s=w.zeta_over_s,
                      alpha_override=w.alpha_override, inlet_n=w.inlet[0], inlet_T=w.inlet[1],
                      inlet_u=tuple(w.inlet[2]))
    s = oracle.init(p, *w.fields())
    oracle.step(s, warmup)
    if steps is None:
        t0 = time.perf_counter()
        oracle.step(s, 2)
        per = (time.perf_counter() - t0) / 2
        steps = max(2, int(budget_s / max(per, 1e-6)))
    t0 = time.perf_counter()
    oracle.step(s, steps)
    el = time.perf_counter() - t0
    return {"value": w.N * steps / el / 1e6, "unit": UNIT, "cores": oracle.get_threads(),
            "kind": "oracle",
            "sample": f"{w.name}: {w.nx}x{w.ny}x{w.nz} cells (the 512x256x256 shock-cloud shrunk 8x "
                      f"per axis), {steps} FP64 steps, {el:.1f} s"}, steps, el


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    base, steps, el = cpu_baseline(steps=args.steps, warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cloud_3d 512x256x256 shock-cloud (oracle on the 64x32x32 "
                                   "sample of the same workload)"},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def l1_fp32_vs_fp64(torch):
    from paper_1302_1125_gb300 import rlb
    from paper_1302_1125_gb300 import workloads as W
    w = W.tube_800()
    out = []
    for prec in (rlb.FP32_STORAGE, rlb.FP64):
        g = rlb.Grid.from_workload(w, precision=prec)
        g.init(*w.fields()).step(w.steps)
        out.append(g.macroscopic(device=False))
        g.close()
    a, b = out
    return {"workload": f"tube_800, {w.steps} steps",
            "n": float(np.abs(a[0] - b[0]).sum() / np.abs(b[0]).sum()),
            "e": float(np.abs(a[1] - b[1]).sum() / np.abs(b[1]).sum()),
            "u_x": float(np.abs(a[2] - b[2]).sum() / np.abs(b[2]).sum())}


def l1_cloud_3d(torch, rlb, W, steps=100):
    """Per-field L1 relative error of the FP32-storage form (both recoveries)
    against the FP64 form on the headline grid itself, 512 x 256 x 256, after
    `steps` steps from the same initial state.  The FP64 form matches the
    FP64 oracle within 1e-10 (tests/test_gpu_parity.py)."""
    w = W.cloud_3d()
    fields = [torch.as_tensor(a, device="cuda") for a in w.fields()]
    out = {}
    for name, prec, rec in (("fp64", rlb.FP64, 0), ("fp32_storage", rlb.FP32_STORAGE, 0),
                            ("fp32_storage_rec64", rlb.FP32_STORAGE, 1)):
        g = rlb.Grid.from_workload(w, precision=prec, recovery_fp64=rec)
        g.init(*fields).step(steps)
        out[name] = g.macroscopic(device=False)
        g.close()
    del fields
    ref = out["fp64"]
    res = {"workload": f"cloud_3d 512x256x256, {steps} steps, against the FP64 form on the same grid",
           "norm": "sum |a - b| / sum |b| per field; u: the velocity vector, sum |u_a - u_b| / sum |u_b|"}
    for name in ("fp32_storage", "fp32_storage_rec64"):
        a = out[name]
        res[name] = {k: float(np.abs(a[i] - ref[i]).sum() / np.abs(ref[i]).sum())
                     for i, k in enumerate(("n", "e", "u_x"))}
        # the velocity as one vector field (u_y, u_z vanish on the symmetry planes)
        res[name]["u"] = float(np.sqrt(((a[2:5] - ref[2:5]) ** 2).sum(0)).sum() /
                               np.sqrt((ref[2:5] ** 2).sum(0)).sum())
    return res


def batch_sweep(torch, rlb, W, hbm_peak, device_index):
    """The 512-tube sweep (seed 1234, each tube 4 Nx steps) in one persistent
    launch with the autotuned shape, and a sample of the same tubes run one by
    one through the single-grid path (FP64 and FP32 storage) for comparison."""
    spec = W.batch_tubes()
    updates = float(np.sum(spec.nx.astype(np.float64) * spec.steps))
    b = rlb.Batch.from_spec(spec)
    b.init(*spec.fields())
    best, trials = b.autotune(spec.steps, divisor=32)
    for _ in range(3):                      # warm-up launches (graph capture included)
        b.step(np.maximum(spec.steps // 64, 1))
    b.init(*spec.fields())
    stream = torch.cuda.current_stream()
    for attempt in range(2):
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(device_index) as cs:
            torch.cuda.synchronize()
            l0 = b.launches
            start.record(stream)
            b.step(spec.steps)
            end.record(stream)
            torch.cuda.synchronize()
        ms = start.elapsed_time(end)
        launches = b.launches - l0
        clk = cs.summary()
        if not rejected(clk):
            break
        b.init(*spec.fields())
    t, ncl = b.tuning()
    b.close()
    value = updates / (ms * 1e-3) / 1e6
    achieved = BYTES_FP32 * updates / (ms * 1e-3) / 1e9

    # the same tubes run separately: every 64th tube by length, Nx steps each
    # (a quarter of the sweep's count; the cost per step does not change)
    order = np.argsort(spec.nx, kind="stable")
    sample = [int(i) for i in order[::64]]
    out = rlb.BC_OUTFLOW, rlb.BC_PERIODIC, rlb.BC_PERIODIC
    sep = {}
    for name, prec in (("fp64", rlb.FP64), ("fp32_storage", rlb.FP32_STORAGE)):
        tot_ms, tot_upd = 0.0, 0.0
        for i in sample:
            o, m = int(spec.offsets[i]), int(spec.nx[i])
            n, T, ux = (a[o:o + m] for a in spec.fields())
            g = rlb.Grid(m, bc_lo=out, bc_hi=out, eta_over_s=float(spec.eta_over_s[i]),
                         zeta_over_s=float(spec.zeta_over_s[i]), dt_over_dx=spec.dt_over_dx,
                         alpha_override=spec.alpha, precision=prec)
            z = np.zeros(m)
            g.init(n, T, ux, z, z)
            g.step(3)
            g.init(n, T, ux, z, z)
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            g.step(m)
            s1.record(stream)
            torch.cuda.synchronize()
            tot_ms += s0.elapsed_time(s1)
            tot_upd += m * float(m)
            g.close()
        sep[name] = {"value": tot_upd / (tot_ms * 1e-3) / 1e6, "unit": UNIT,
                     "sample": f"{len(sample)} of the 512 tubes (every 64th by length), Nx steps each "
                               f"({tot_upd:.3g} cell updates), each alone through rlb_create/rlb_step, "
                               f"one launch per step"}
    # the same sweep under the exact 1-D symmetry reduction (7 classes per
    # distribution), reported beside, not instead of, the 19-population number
    br = rlb.Batch.from_spec(spec, symmetry_1d=1)
    br.init(*spec.fields())
    best_r, _ = br.autotune(spec.steps, divisor=32)
    for _ in range(3):
        br.step(np.maximum(spec.steps // 64, 1))
    br.init(*spec.fields())
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    r0.record(stream)
    br.step(spec.steps)
    r1.record(stream)
    torch.cuda.synchronize()
    ms_r = r0.elapsed_time(r1)
    tr, _ = br.tuning()
    br.close()
    reduced = {"value": updates / (ms_r * 1e-3) / 1e6, "unit": UNIT, "ms": ms_r,
               "bytes_per_update": BYTES_SYM1D,
               "hbm_equiv_gbs": BYTES_SYM1D * updates / (ms_r * 1e-3) / 1e9,
               "tuning": {k: v for k, v in tr.as_dict().items() if k != "ms"},
               "what": "symmetry_1d: 7 population classes per distribution (exact for 1-D tubes with "
                       "u_y = u_z = 0); cell updates counted as for the 19-population step"}
    return {"workload": "batch_tubes: 512 1-D shock tubes from seed 1234, Nx log-uniform in [256, 8192], "
                        "eta/s U[0.01, 0.5], pressure ratio log-U[2, 40], gamma_L U[1, 1.5], alpha 0.2, "
                        "dt/dx 0.15, each tube 4 Nx steps, FP32 storage",
            "tubes": int(spec.B), "cells": int(spec.offsets[-1]), "cell_updates": updates,
            "value": value, "unit": UNIT, "ms": ms, "gpu_launches": launches,
            "tuning": {k: v for k, v in t.as_dict().items() if k != "ms"}, "resident_clusters": ncl,
            "autotune_trials": len(trials),
            "roofline": issue_roofline(profiled_value("tubes_kernel_batch_512.md",
                                                      "thread_instructions_per_update"),
                                       value * 1e6, clk,
                                       "instruction issue: the tubes in flight are L2-resident (98 % hit "
                                       "rate), so HBM does not bound the batch; thread-instructions per "
                                       "cell update from the committed ncu capture"),
            "hbm_equiv": {"achieved": achieved, "unit": "GB/s", "bytes_per_update": BYTES_FP32,
                          "note": "algorithmic bytes / time, for comparison with the grid form only"},
            "separate_runs": sep,
            "batched_over_separate_fp64": value / sep["fp64"]["value"],
            "symmetry_1d": reduced,
            "clocks": clk}


def sphere_run(torch, rlb, W, device_index):
    """The paper's own 3-D run (Sec. III): 200 x 100 x 100 cells with a solid
    sphere held at the ambient equilibrium, beta ~ 0.2 shock, viscous
    (tau = 1); FP32 storage for all 1000 steps, FP64 for 100."""
    w = W.sphere_cloud("beta02", viscous=True)
    fields = [torch.as_tensor(a, device="cuda") for a in w.fields()]
    out = {"workload": "sphere_cloud: the paper's 3-D shock-cloud run, 200x100x100, solid sphere r=10 at "
                       "(100,50,50) held at (n1, T1, u=0), slab x<=65 at T0=2.71 T1, n0=0.9 n1, inlet at x=0, "
                       "open faces, tau=1, alpha 0.2, dt/dx 0.15",
           "cells": w.N, "solid_cells": int(w.solid_mask().sum()), "unit": UNIT}
    stream = torch.cuda.current_stream()
    for name, prec, steps in (("fp32_storage", rlb.FP32_STORAGE, w.steps), ("fp64", rlb.FP64, 100)):
        g = rlb.Grid.from_workload(w, precision=prec)
        g.init(*fields)
        g.set_solid(w.solid_mask(), w.solid[1], w.solid[2])
        g.step(3)
        g.init(*fields)
        g.set_solid(w.solid_mask(), w.solid[1], w.solid[2])
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = g.launches
        s0.record(stream)
        g.step(steps)
        s1.record(stream)
        torch.cuda.synchronize()
        ms = s0.elapsed_time(s1)
        out[name] = {"value": w.N * steps / (ms * 1e-3) / 1e6, "steps": steps, "ms_per_step": ms / steps,
                     "gpu_launches": g.launches - l0}
        g.close()
    return out


def cloud_2d_run(torch, rlb, W, hbm_peak, steps=200):
    """The 2-D shock-cloud, 2048 x 1024 (FP32 storage): the 19-population step
    and the exact 2-D symmetry reduction (u_z = 0: 14 class planes per
    distribution), timed separately, and their L1 difference after the timed
    steps (the rounding order of the moment sums only)."""
    w = W.cloud_2d()
    fields = [torch.as_tensor(a, device="cuda") for a in w.fields()]
    stream = torch.cuda.current_stream()
    out = {"workload": f"cloud_2d: 2-D shock-cloud {w.nx}x{w.ny} (inlet at x=0, outflow at x=Nx, periodic y; "
                       f"cloud r=96 at (700,512), density x10, pressure balanced); eta/s {w.eta_over_s}, "
                       f"dt/dx {w.dt_over_dx}; {steps} timed steps; inputs larger than L2",
           "cells": w.N, "unit": UNIT}
    macro = {}
    for name, sym, nbytes in (("fp32_storage", 0, BYTES_FP32), ("symmetry_2d", 1, BYTES_SYM2D)):
        g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, symmetry_2d=sym)
        g.init(*fields)
        g.step(3)
        g.init(*fields)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = g.launches
        s0.record(stream)
        g.step(steps)
        s1.record(stream)
        torch.cuda.synchronize()
        ms = s0.elapsed_time(s1)
        launches = g.launches - l0
        macro[name] = g.macroscopic(device=False)
        g.close()
        mlups = w.N * steps / (ms * 1e-3) / 1e6
        gbs = nbytes * mlups * 1e6 / 1e9
        out[name] = {"value": mlups, "ms_per_step": ms / steps, "bytes_per_update": nbytes,
                     "hbm_equiv_gbs": gbs, "hbm_frac": gbs / hbm_peak, "gpu_launches": launches}
    a, b = macro["symmetry_2d"], macro["fp32_storage"]
    out["symmetry_2d"]["l1_vs_19_populations"] = {
        "n": float(np.abs(a[0] - b[0]).sum() / np.abs(b[0]).sum()),
        "e": float(np.abs(a[1] - b[1]).sum() / np.abs(b[1]).sum()),
        "u_x": float(np.abs(a[2] - b[2]).sum() / np.abs(b[5]).sum())}
    out["symmetry_2d"]["what"] = ("symmetry_2d: 14 population classes per distribution (exact for nz = 1 and "
                                  "u_z = 0); cell updates counted as for the 19-population step")
    return out


PAPER_TUBES = [
    ("P ratio 5.43/2.22, T ratio 2, eta/s 0.1, alpha 0 (beta ~ 0.2)", 5.43 / 2.22, 0.1, 0.0, 220.0),
    ("P ratio 32, T ratio 2, eta/s 0.01, alpha 0.15, extended model (beta ~ 0.7)", 32.0, 0.01, 0.15, 1069.0),
]


def cpu_baseline_paper_tubes(W):
    """Part of the CPU baseline: the oracle, as it stands, on the paper's timed
    1-D runs (the cases of PAPER_TUBES, 1600 steps each, init and
    macroscopic output included) on all host cores."""
    import oracle
    oracle.set_threads(os.cpu_count() or 1)
    out = []
    for _desc, ratio, eta, alpha, _paper_ms in PAPER_TUBES:
        host = [np.ascontiguousarray(a) for a in W.riemann_tube(800, ratio, 2.0, eta_over_s=eta).fields()]
        p = oracle.Params(nx=800, dt=0.25, eta_over_s=eta, alpha_override=alpha)
        t0 = time.perf_counter()
        st = oracle.init(p, *host)
        oracle.step(st, 1600)
        oracle.macroscopic(st)
        out.append({"oracle_ms": 1e3 * (time.perf_counter() - t0), "oracle_cores": oracle.get_threads(),
                    "oracle_nonphysical_cells": int(st.nonphysical)})
    return out


def paper_runs(torch, rlb, W):
    """The paper's timed 1-D runs (Sec. III: 800 cells, dt/dx 0.25, t = 3.2 fm,
    i.e. 1600 steps), each as a whole run through the public API with host
    arrays: rlb_init from host fields, the steps, rlb_macroscopic to host.
    Next to them the paper's own wall times (an unnamed "standard PC";
    context only); the oracle's times on the same runs come from
    cpu_baseline_paper_tubes."""
    out = {"what": "the paper's timed 1-D runs: 800 cells, dt/dx 0.25, 1600 steps; wall time of the whole run "
                   "(init from host, steps, macroscopic output to host); median of 3",
           "runs": []}
    for desc, ratio, eta, alpha, paper_ms in PAPER_TUBES:
        w = W.riemann_tube(800, ratio, 2.0, eta_over_s=eta)
        host = [np.ascontiguousarray(a) for a in w.fields()]
        outbuf = np.empty((6, w.N))
        res = {"workload": desc, "steps": 1600, "paper_ms": paper_ms,
               "paper_hardware": "an unnamed 'standard PC' CPU (core count and precision not stated)"}
        for key, prec, sym in (("fp64_ms", rlb.FP64, 0), ("fp32_ms", rlb.FP32_STORAGE, 0),
                               ("fp32_symmetry_1d_ms", rlb.FP32_STORAGE, 1)):
            g = rlb.Grid(w.nx, bc_lo=w.bc_lo, bc_hi=w.bc_hi, eta_over_s=eta, dt_over_dx=0.25,
                         alpha_override=alpha, precision=prec, symmetry_1d=sym)
            g.init(*host).step(10)
            times = []
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                g.init(*host)
                g.step(1600)
                rlb.rlb_macroscopic(g.ctx, outbuf, 0)
                torch.cuda.synchronize()
                times.append(1e3 * (time.perf_counter() - t0))
            g.close()
            res[key] = sorted(times)[1]
        out["runs"].append(res)
    return out


def basic_model_run(torch, rlb, W, hbm_peak):
    """The basic model (Sec. II: D3Q19 with unit diagonals) on the headline
    grid, and the paper's basic-versus-extended comparison (P ratio 32,
    beta ~ 0.7, eta/s 0.01, dt/dx 0.25; alpha 0.15 for the extended model)."""
    w = W.cloud_3d()
    fields = [torch.as_tensor(a, device="cuda") for a in w.fields()]
    stream = torch.cuda.current_stream()
    out = {"workload": "cloud_3d 512x256x256 on the basic lattice (alpha 0.2, dt/dx 0.15)", "unit": UNIT}
    for name, prec, steps in (("fp32_storage", rlb.FP32_STORAGE, 50), ("fp64", rlb.FP64, 5)):
        g = rlb.Grid(w.nx, w.ny, w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, inlet=w.inlet, eta_over_s=w.eta_over_s,
                     zeta_over_s=w.zeta_over_s, dt_over_dx=w.dt_over_dx, alpha_override=w.alpha_override,
                     precision=prec, model=rlb.MODEL_BASIC)
        g.init(*fields)
        try:
            g.step(3)
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            g.step(steps)
            s1.record(stream)
            torch.cuda.synchronize()
        except rlb.RLBError as e:
            out[name] = {"value": None, "status": rlb.status_string(e.status)}
            g.close()
            continue
        ms = s0.elapsed_time(s1) / steps
        bytes_ = BYTES_FP32 if prec == rlb.FP32_STORAGE else BYTES_FP64
        out[name] = {"value": w.N / (ms * 1e-3) / 1e6, "ms_per_step": ms, "steps": steps,
                     "hbm_frac": bytes_ * w.N / (ms * 1e-3) / 1e9 / hbm_peak}
        g.close()
    del fields
    cmp = {}
    for name, model, alpha in (("basic", rlb.MODEL_BASIC, 0.0), ("extended", rlb.MODEL_EXTENDED, 0.15)):
        t = W.riemann_tube(800, 32.0, 2.0, eta_over_s=0.01, dt_over_dx=0.25, alpha_override=alpha)
        g = rlb.Grid(t.nx, eta_over_s=0.01, dt_over_dx=0.25, alpha_override=alpha, precision=rlb.FP64,
                     model=model)
        g.init(*t.fields())
        done, status = 0, "physical after 1200 steps"
        while done < 1200:
            try:
                g.step(50)
            except rlb.RLBError as e:
                status = f"{rlb.status_string(e.status)} within steps {done + 1}-{done + 50}"
                break
            done += 50
        cmp[name] = status
        g.close()
    out["paper_comparison_beta07"] = {"setup": "800-cell tube, P ratio 32, eta/s 0.01, dt/dx 0.25, FP64; "
                                               "alpha 0 (basic), 0.15 (extended)", **cmp}
    return out


def run_ours(args):
    global _dist
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        _dist = dist
    else:
        torch.cuda.set_device(0)
    from paper_1302_1125_gb300 import build as B
    B.build()
    from paper_1302_1125_gb300 import rlb
    from paper_1302_1125_gb300 import workloads as W

    hbm_peak, peak_kind = peaks()
    w = W.cloud_3d()
    N = w.N
    fields = w.fields()
    dev_fields = [torch.as_tensor(a, device="cuda") for a in fields]

    # FP32-storage form (the headline)
    g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE)
    g.init(*dev_fields)
    kernel = g.step_kernel
    ms, clk, launches, window = timed_steps(torch, g, args.steps, args.warmup, local, window_s=2.0)
    ms = max_over_ranks(torch, ms)
    per_step = ms / args.steps
    value = job_value(world, N * args.steps, ms * 1e-3)
    achieved = BYTES_FP32 * N / (per_step * 1e-3) / 1e9
    g.close()

    # the same form with the block staging each population's stencil tile by
    # bulk copies (thread_mapping 3), in place of each thread staging its own
    gs = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, thread_mapping=rlb.MAPPING_BULK_TILES)
    gs.init(*dev_fields)
    mss, _, _, _ = timed_steps(torch, gs, args.steps, args.warmup, local)
    mss = max_over_ranks(torch, mss)
    value_s = job_value(world, N * args.steps, mss * 1e-3)
    kernel_s = gs.step_kernel
    gs.close()

    # the same form with its Landau-frame recovery in FP64 (recovery_fp64)
    gr = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, recovery_fp64=1)
    gr.init(*dev_fields)
    msr, clkr, _, _ = timed_steps(torch, gr, args.steps, args.warmup, local)
    msr = max_over_ranks(torch, msr)
    value_r = job_value(world, N * args.steps, msr * 1e-3)
    gr.close()

    # FP64 form on the same grid
    g64 = rlb.Grid.from_workload(w, precision=rlb.FP64)
    g64.init(*dev_fields)
    k64 = max(3, args.steps // 10)
    ms64, clk64, _, _ = timed_steps(torch, g64, k64, max(3, args.warmup), local)
    ms64 = max_over_ranks(torch, ms64)
    value64 = world * N * k64 / (ms64 * 1e-3) / 1e6
    ach64 = BYTES_FP64 * N / (ms64 / k64 * 1e-3) / 1e9
    g64.close()
    del dev_fields

    # end to end through the public API with host buffers: pinned host fields
    # -> rlb_init -> K steps -> rlb_macroscopic into pinned host memory
    host_in = [torch.from_numpy(a).pin_memory() for a in fields]
    host_out = torch.empty((6, N), dtype=torch.float64).pin_memory()
    ge = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE)
    ge.init(*[a.numpy() for a in host_in]).step(args.warmup)
    torch.cuda.synchronize()
    # three runs, the median reported: the host copies share the host's
    # memory bandwidth with other work and vary from run to run.  Each call
    # returns after its work (rlb_init, rlb_step and rlb_macroscopic
    # synchronise), so the wall clock splits into the three phases.
    runs = []
    with ClockSampler(local) as cs_e2e:
        for _ in range(3):
            barrier()
            t0 = time.perf_counter()
            ge.init(*[a.numpy() for a in host_in])
            t1 = time.perf_counter()
            ge.step(args.steps)
            t2 = time.perf_counter()
            rlb.rlb_macroscopic(ge.ctx, host_out.numpy(), 0)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            runs.append((max_over_ranks(torch, t3 - t0), t1 - t0, t2 - t1, t3 - t2))
    barrier()
    ge.close()
    e2e_s, ti, ts, to = sorted(runs)[1]
    e2e = {"value": world * N * args.steps / e2e_s / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": 5 * 8 * N / args.steps, "d2h_bytes_per_step": 6 * 8 * N / args.steps,
           "what": "pinned host n,T,u -> rlb_init -> K steps -> rlb_macroscopic to pinned host; median of 3 runs",
           "runs_ms": [1e3 * r[0] for r in runs],
           "phases_ms": {"init_from_host": 1e3 * ti, "steps": 1e3 * ts, "output_to_host": 1e3 * to},
           "clocks": cs_e2e.summary()}

    batch = batch_sweep(torch, rlb, W, hbm_peak, local) if not args.no_batch else None
    sphere = sphere_run(torch, rlb, W, local) if not args.no_batch else None
    cloud2d = cloud_2d_run(torch, rlb, W, hbm_peak) if not args.no_batch else None
    paper = paper_runs(torch, rlb, W) if not args.no_batch and (world == 1 or rank == 0) else None
    basic = basic_model_run(torch, rlb, W, hbm_peak) if not args.no_batch else None
    l1_headline = l1_cloud_3d(torch, rlb, W) if not args.no_batch else None
    if rank != 0:
        return 0
    l1 = l1_fp32_vs_fp64(torch)
    base = cpu_baseline()[0] if world == 1 or rank == 0 else None
    if paper is not None:
        for run, orc_time in zip(paper["runs"], cpu_baseline_paper_tubes(W)):
            run.update(orc_time)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "cloud_3d: 3-D shock-cloud 512x256x256 (slab-driven shock, pressure "
                               "ratio 10; cloud r=48 at (180,128,128), density x10, pressure balanced); "
                               "eta/s 0.05, alpha 0.2, dt/dx 0.15",
                   "cells": N,
                   "precision": "FP32 populations (stored, streamed, relaxed in FP32); moment sums and "
                                "E^2-|M|^2 in double-float (float pairs, error-free TwoSum/FMA); the rest of "
                                "the Landau-frame recovery, tau and the equilibrium coefficients in FP32; no FP64 "
                                "instruction",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2: 10.2 GB of populations read+written per step"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak,
                     "traffic": profiled_traffic("step_kernel_fp32_cloud_3d.md", N),
                     "note": f"{BYTES_FP32} algorithmic bytes per cell update x {N} cells per launch "
                             f"/ CUDA-event time per launch; peak {peak_kind} copy bandwidth"},
        "issue": issue_roofline(profiled_value("step_kernel_fp32_cloud_3d.md", "thread_instructions_per_cell"),
                                value * 1e6 / world, clk,
                                "instruction issue of the headline kernel; thread-instructions per cell from the "
                                "committed ncu capture"),
        "clock_window": window,
        "step_kernel": kernel,
        "fp32_bulk_staging": {"value": value_s, "unit": UNIT, "ms_per_step": mss / args.steps,
                              "hbm_frac": BYTES_FP32 * N / (mss / args.steps * 1e-3) / 1e9 / hbm_peak,
                              "step_kernel": kernel_s,
                              "what": "the same FP32-storage step with each population's stencil tile staged "
                                      "into shared memory by block-wide bulk copies (tensor-map boxes, "
                                      "cp.async.bulk.tensor, on mbarriers; thread_mapping 3)"},
        "fp32_rec64": {"value": value_r, "unit": UNIT, "ms_per_step": msr / args.steps,
                       "hbm_frac": BYTES_FP32 * N / (msr / args.steps * 1e-3) / 1e9 / hbm_peak,
                       "precision": "FP32 populations, double-float moment sums, Landau-frame recovery of both "
                                    "time levels in FP64 (rlb_options.recovery_fp64 = 1)",
                       "alu": alu_roofline(profiled_value("step_kernel_fp32_rec64_cloud_3d.md", "dp_thread_ops_per_cell"),
                                           value_r * 1e6 / world, N_SM * DP_LANES_PER_SM, clkr,
                                           "FP64 pipe: the recovery's DP thread-operations per cell (committed ncu "
                                           "capture) x cells per second, against 152 SMs x 2 FP64 lanes x the "
                                           "sampled SM clock"),
                       "clocks": clkr},
        "fp64_form": {"value": value64, "unit": UNIT, "steps": k64, "ms_per_step": ms64 / k64,
                      "hbm_achieved_gbs": ach64, "hbm_frac": ach64 / hbm_peak,
                      "alu": alu_roofline(profiled_value("step_kernel_fp64_cloud_3d.md", "dp_thread_ops_per_cell"),
                                          value64 * 1e6 / world, N_SM * DP_LANES_PER_SM, clk64,
                                          "FP64 pipe: DP thread-operations per cell (committed ncu capture) x "
                                          "cells per second, against 152 SMs x 2 FP64 lanes x the sampled SM "
                                          "clock"),
                      "clocks": clk64},
        "fp32_over_fp64": value / value64,
        "l1_error_headline": l1_headline,
        "l1_error_fp32_vs_fp64": l1,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": base,
        "batch": batch,
        "sphere_cloud": sphere,
        "cloud_2d": cloud2d,
        "paper_runs": paper,
        "basic_model": basic,
    }
    print(json.dumps(line), flush=True)
    if _dist is not None:
        _dist.destroy_process_group()
    return 0


def arg_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched sweep, the sphere-cloud run and the basic-model runs")
    return ap


def main():
    args = arg_parser().parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
