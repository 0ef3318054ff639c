"""Benchmark: layer-cell-updates per second of the two-layer shallow-water step on GB300.

Workload (default): the 2048 x 2048 fixed-grid shelf problem, two layers, FP64,
second order with the MC limiter, walls on all sides; one benchmark step is one
full time step of the level (x sweep + y sweep, all cells). Inputs are larger
than L2 (201 MB of state per buffer), so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mlswe|reference]

``--impl reference`` times the FP64 CPU oracle (the plain reference
implementation) on the host cores for the same workload and metric.
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1803_01450_gb300 import inputs as I  # noqa: E402

METRIC = "layer-cell-updates/s (FP64, 1 GB300) batched vs per-patch; adjoint/forward cost"
UNIT = "LCU/s"
N_CELLS = 2048
M_LAYERS = 2

# FP64 operations per cell update of the step kernels (x sweep + y sweep), counted by ncu
# on the scale workload (2 * dfma + dadd + dmul instructions, thread level), with the
# halo edges of each tile removed. See profiles/ for the capture.
FP64_FLOP_PER_CELL_UPDATE = None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return rank, ws


def run_reference(args):
    """The FP64 CPU oracle on the host cores, same workload and metric."""
    rank, ws = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = I.scale(N_CELLS)
    P = oracle.params(M=2, dry_tol=w["dry_tol"])
    q, B = w["q"], w["B"]
    dt = 0.9 * w["dx"] / 205.0
    for _ in range(args.warmup):
        q, _, _ = oracle.step_walled(P, q, B, w["dx"], w["dy"], dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q, _, _ = oracle.step_walled(P, q, B, w["dx"], w["dy"], dt)
    el = time.perf_counter() - t0
    lcu = N_CELLS * N_CELLS * M_LAYERS * args.steps
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    v = lcu / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "scale: 2048x2048 fixed grid, 2 layers, shelf bathymetry, 8 humps, order 2 MC",
                       "cells": N_CELLS * N_CELLS, "layers": M_LAYERS},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full steps of the 2048^2 workload after {args.warmup} warm-up"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(seconds_budget=15.0):
    """Oracle throughput on the host cores over a bounded sample of the same workload."""
    import oracle
    oracle.build()
    w = I.scale(N_CELLS)
    P = oracle.params(M=2, dry_tol=w["dry_tol"])
    q, B = w["q"], w["B"]
    dt = 0.9 * w["dx"] / 205.0
    t0 = time.perf_counter()
    n = 0
    while True:
        q, _, _ = oracle.step_walled(P, q, B, w["dx"], w["dy"], dt)
        n += 1
        if time.perf_counter() - t0 > seconds_budget or n >= 20:
            break
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": N_CELLS * N_CELLS * M_LAYERS * n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} full time steps of the 2048^2 scale workload ({el:.1f} s)"}


def run_gpu(args):
    import torch
    import paper_1803_01450_gb300 as pkg

    rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    pkg.build()

    w = I.scale(N_CELLS, seed=1000 + rank)
    cfg = pkg.Config(M=2, dry_tol=w["dry_tol"], order=2, limiter=2, max_levels=1)
    stream = torch.cuda.Stream(device=dev)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1e5, 1e5, N_CELLS, N_CELLS)], stream=stream.cuda_stream)
    H.set_bathymetry(0, w["B"])
    H.set_state(0, 0, w["q"])
    dt = 0.9 * w["dx"] / 205.0
    H.set_dt(0, dt)
    for _ in range(args.warmup):
        H.step_level(0)
    torch.cuda.synchronize()

    # ---- device-timed region: K steps, inputs resident in HBM ----
    H.timing(enable=True)
    clk = ClockSampler(local)
    clk.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        H.step_level(0)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    clocks = clk.stop()
    per_kernel, total_launches = H.timing(enable=False)

    # ---- end-to-end through the public API with host buffers ----
    import torch as _t
    qh = _t.empty(w["q"].shape, dtype=_t.float64, pin_memory=True).numpy()
    qh[...] = w["q"]
    xy = np.stack([np.linspace(1e4, 9e4, 32), np.linspace(2e4, 8e4, 32)], axis=1)
    e2e_steps = max(3, min(args.steps, 10))
    H.set_state(0, 0, qh)
    H.step_level(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        H.set_state(0, 0, qh)
        H.step_level(0)
        g = H.read_gauges(0, xy) if hasattr(H, "read_gauges") else None
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    H.close()

    lcu_per_step = N_CELLS * N_CELLS * M_LAYERS
    tmax = ms
    if ws > 1:
        tt = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        tmax = float(tt.item())
    value = lcu_per_step * args.steps * ws / (tmax * 1e-3)

    peaks = _peaks()
    sx_ms, sx_n = per_kernel["sweep_x"]
    sy_ms, sy_n = per_kernel["sweep_y"]
    roof = None
    if FP64_FLOP_PER_CELL_UPDATE:
        step_ms = (sx_ms + sy_ms) / max(1, sx_n)
        ach = FP64_FLOP_PER_CELL_UPDATE * N_CELLS * N_CELLS / (step_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": 1.012, "unit": "TFLOP/s", "frac": ach / 1.012,
                "traffic": None}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "scale: 2048x2048 fixed grid, 2 layers, shelf bathymetry, 8 humps, order 2 MC",
                   "cells": N_CELLS * N_CELLS, "layers": M_LAYERS, "l2": "inputs larger than L2 (201 MB state)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "clocks": clocks,
        "gpu_launches": total_launches,
        "kernels_ms_per_launch": {k: (v[0] / v[1] if v[1] else None) for k, v in per_kernel.items() if v[1]},
        "roofline": roof,
        "e2e": {"value": lcu_per_step * e2e_steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(w["q"].nbytes + xy.nbytes), "d2h_bytes_per_step": 32 * M_LAYERS * 8},
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mlswe", choices=["mlswe", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
