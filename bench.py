"""Benchmark: layer-cell-updates per second of the two-layer shallow-water AMR hot path on GB300.

Headline workload (``value``): the 2048 x 2048 fixed-grid shelf problem (two layers, FP64,
second order with the MC limiter, walls on all sides); one benchmark step is one full time
step of the level (x sweep + y sweep over every cell). The state (201 MB per buffer) is
larger than L2, so no flush is needed between steps.

Also reported on the same line:
  * ``batched_amr``: three levels (512^2 coarse, ratios 4 and 4) over the shore bathymetry
    with 1000 level-1 and 3000 level-2 patches of sides 16..64 (seeded synthetic layout),
    whole subcycled coarse steps; all patches of a level in one persistent launch replayed
    from a CUDA graph versus one launch per patch;
  * ``ensemble``: 256 members of sizes U{128..512}^2 with a refined level (ratio 4), all
    members stepped together with per-member time steps, batched versus per-patch;
  * ``adjoint``: gauge-misfit gradient on a 512^2 grid over 200 first-order steps with a
    checkpoint every 20 steps: backward (recomputation + transposed steps) over forward;
  * ``three_layers``: the headline workload with three layers (general M-layer solver).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mlswe|reference]

``--impl reference`` times the FP64 CPU oracle (the plain reference implementation) on the
host cores for the headline workload and metric. Prints one JSON line.
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

# FP64 operations per cell update of the method (x sweep + y sweep, order 2, MC limiter,
# eigenvalue guesses + 2 Newton steps), counted by the oracle's counting scalar on the
# headline workload: `python -m oracle.count_flops`. Half of it belongs to each sweep.
FP64_FLOP_PER_CELL_UPDATE = 1293.25
# The same count for the three-layer version of the workload (inputs.scale3).
FP64_FLOP_PER_CELL_UPDATE_3 = 4134.82
# ... and for the four-layer version (inputs.scale4).
FP64_FLOP_PER_CELL_UPDATE_4 = 10523.35
# The unsplit step (transverse Riemann solves) on the same workload, per cell update: each edge
# pass (x edges, y edges) and the transverse correction fluxes plus the update.
FP64_FLOP_PER_CELL_UPDATE_UNSPLIT = 2456.89
FP64_FLOP_UNSPLIT_EDGE_PASS = 1143.94
FP64_FLOP_PER_CELL_UPDATE_UNSPLIT_3 = 6816.15  # three layers (inputs.scale3)
def _measured_hbm_gbs(default=6674.8):
    """HBM copy bandwidth measured on the GB300s (STREAM-style copy), from the peaks
    file the machine provides; the earlier measurement when the file is absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return default


HBM_PEAK_GBS = _measured_hbm_gbs()
# FP64 peak derived from the unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes per launch of the x sweep on the headline workload (ncu, see profiles/); None
# while the kernel has changed since the last capture.
SWEEP_X_DRAM_BYTES = 401.5e6


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
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def replica_seed(rank: int) -> int:
    """Seed of the headline replica a rank advances (independent problems, one per rank)."""
    return 1000 + rank


def max_over_ranks(ms: float, ws: int, device=None) -> float:
    """Longest timed-region duration over all ranks (every rank receives it)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_step_per_rank: float, steps: int, ws: int, tmax_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_step_per_rank * steps * ws / (tmax_ms * 1e-3)


def _workload_name():
    return "scale: 2048x2048 fixed grid, 2 layers, shelf bathymetry, 8 humps, order 2 MC, walls"


def run_reference(args):
    """The FP64 CPU oracle on the host cores, same workload and metric (rank 0 only)."""
    rank, ws = _dist()
    if rank != 0:
        return
    import oracle
    oracle.use_timing_build()
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
    cores = oracle.threads()
    v = N_CELLS * N_CELLS * M_LAYERS * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_name(), "cells": N_CELLS * N_CELLS, "layers": M_LAYERS},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full time steps of the 2048^2 workload after "
                                       f"{args.warmup} warm-up steps, oracle built -O3 (scheduled for Neoverse V2 on "
                                       f"Arm hosts), OpenMP over rows",
                             "host_cores": _host_cores()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _host_cores():
    """Logical CPUs, those this process may run on, and physical cores (distinct (package,
    core) pairs in sysfs; None where the topology is not readable)."""
    phys = set()
    base = "/sys/devices/system/cpu"
    try:
        for d in os.listdir(base):
            if d.startswith("cpu") and d[3:].isdigit():
                t = os.path.join(base, d, "topology")
                with open(os.path.join(t, "core_id")) as f:
                    core = f.read().strip()
                with open(os.path.join(t, "physical_package_id")) as f:
                    pkg = f.read().strip()
                phys.add((pkg, core))
    except OSError:
        phys = set()
    return {"logical": os.cpu_count(), "affinity": len(os.sched_getaffinity(0)),
            "physical": len(phys) or None}


def _oracle_rate(seconds_budget, max_steps):
    """LCU/s of the oracle's timing build over whole headline time steps (about seconds_budget
    of work, at least one step), and the OpenMP threads it ran with."""
    import oracle
    oracle.use_timing_build()
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
        if time.perf_counter() - t0 > seconds_budget or n >= max_steps:
            break
    el = time.perf_counter() - t0
    return N_CELLS * N_CELLS * M_LAYERS * n / el, n, el, oracle.threads()


def cpu_baseline(seconds_budget=12.0):
    """Oracle throughput on the host cores over a bounded sample of the headline workload
    (whole time steps, about seconds_budget of work), with every core the process may use and
    with one thread (a child process with OMP_NUM_THREADS=1, about 8 s)."""
    v, n, el, threads = _oracle_rate(seconds_budget, 400)
    one = None
    try:
        code = ("import json, bench; r = bench._oracle_rate(8.0, 3); "
                "print(json.dumps({'value': r[0], 'steps': r[1], 's': r[2], 'threads': r[3]}))")
        env = dict(os.environ, OMP_NUM_THREADS="1")
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=300)
        if out.returncode == 0:
            one = json.loads(out.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError):
        one = None
    return {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} full time steps of the 2048^2 headline workload ({el:.1f} s), oracle built -O3 "
                      f"(scheduled for Neoverse V2 on Arm hosts), OpenMP over rows",
            "host_cores": _host_cores(),
            "one_core": None if one is None else {"value": one["value"], "threads": one["threads"],
                                                  "sample": f"{one['steps']} full time steps ({one['s']:.1f} s)"}}


def _interior_updates(H, member_count, levels, ratios):
    """Cell updates of one coarse step (patch cells x time steps of each level)."""
    tot = 0
    for m in range(member_count):
        steps = 1
        for l in range(levels):
            if l > 0:
                steps *= ratios[l - 1]
            boxes = H.get_patches(m, l)
            tot += steps * int(sum((b[2] - b[0]) * (b[3] - b[1]) for b in boxes))
    return tot


def _time_advance(torch, H, stream, n_steps):
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    H.advance(n_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _amr_transfer_bytes(H, n0, r, M):
    """Algorithmic bytes of one coarse step's level transfers on a 3-level layout (ratios r, r):
    ghost fill (A7 with the refinement of A10): per ring cell of a refined patch (two cells
    wide, once even where rings overlap) its 3M values written and its fine B read, plus the
    coarse cells under the ring and their face neighbours read at two time levels with B;
    coarsening (A11): every covered coarse cell reads its r^2 fine cells and writes itself;
    reflux (A12): every coarse/fine edge reads the coarse and the r fine mass fluxes and
    updates the uncovered cell's depths. Counts per level step times level steps per coarse
    step (r on level 1, r^2 on level 2; transfers onto level l once per level-l step)."""
    import scipy.ndimage as nd
    F = 3 * M
    shapes = [n0, n0 * r, n0 * r * r]
    masks = [np.ones((n0, n0), bool)]
    for l in (1, 2):
        m = np.zeros((shapes[l], shapes[l]), bool)
        for (i0, j0, i1, j1) in H.get_patches(0, l).tolist():
            m[j0:j1, i0:i1] = True
        masks.append(m)
    cross = np.array([[0, 1, 0], [1, 1, 1], [0, 1, 0]], bool)
    ghost = avg = refl = 0
    for l in (1, 2):
        m, nc = masks[l], shapes[l - 1]
        ring = nd.binary_dilation(m, structure=np.ones((5, 5), bool)) & ~m
        under = nd.binary_dilation(ring.reshape(nc, r, nc, r).any(axis=(1, 3)), structure=cross)
        ghost += (int(ring.sum()) * (F + 1) * 8 + int(under.sum()) * (2 * F + 1) * 8) * r ** l
        cov = m.reshape(nc, r, nc, r).any(axis=(1, 3))
        avg += int(cov.sum()) * F * (r * r + 1) * 8 * r ** (l - 1)
        inp = masks[l - 1]
        ex = (cov[:, 1:] != cov[:, :-1]) & np.where(cov[:, 1:], inp[:, :-1], inp[:, 1:])
        ey = (cov[1:, :] != cov[:-1, :]) & np.where(cov[1:, :], inp[:-1, :], inp[1:, :])
        refl += (int(ex.sum()) + int(ey.sum())) * M * (3 + r) * 8 * r ** (l - 1)
    return {"ghost_fill": ghost, "average": avg, "reflux": refl}


def bench_batched_amr(pkg, torch, stream, steps=3, n0=512, patches=(1000, 3000)):
    """Three-level AMR over the shore bathymetry, 1000 + 3000 synthetic patches (the figure;
    smaller coarse grids and patch counts give short cases of the same kernels for profiling);
    then the level transfers per kernel class and one regrid (flag tolerance 5e-5: the humps'
    slopes are about 1e-4, so the regrid refines around them)."""
    r = 4
    H, chosen, upd = _batched_amr_hierarchy(pkg, stream, n0, patches)
    n_patches = [len(H.get_patches(0, l)) for l in (1, 2)]
    H.advance(1)
    ms_b = _time_advance(torch, H, stream, steps)
    H.set_execution(use_graphs=False, per_patch_launches=True)
    H.advance(1)
    ms_p = _time_advance(torch, H, stream, max(1, steps // 2))
    H.set_execution(use_graphs=True, per_patch_launches=False)
    # level transfers of further coarse steps, timed per kernel class (direct launches)
    H.timing(enable=True)
    H.advance(steps)
    torch.cuda.synchronize()
    per, _ = H.timing(enable=False)
    tb = _amr_transfer_bytes(H, n0, r, M_LAYERS)
    transfers = {}
    for k in ("ghost_fill", "average", "reflux"):
        ms_k = per[k][0] / steps
        gbs = tb[k] / (ms_k * 1e-3) / 1e9
        transfers[k] = {"ms_per_coarse_step": ms_k, "launches_per_coarse_step": per[k][1] / steps,
                        "algorithmic_bytes_per_coarse_step": tb[k], "achieved_gbs": gbs,
                        "frac_of_hbm": gbs / HBM_PEAK_GBS}
    transfers["sweeps_ms_per_coarse_step"] = (per["sweep_x"][0] + per["sweep_y"][0]) / steps
    # one regrid (A8 flags + clustering, A10 refinement of the new patches)
    old = [H.get_patches(0, l) for l in (1, 2)]
    H.timing(enable=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H.regrid(0)
    torch.cuda.synchronize()
    regrid_s = time.perf_counter() - t0
    per, _ = H.timing(enable=False)
    flag_cells = n0 * n0 + (n0 * r) ** 2
    fb = flag_cells * ((M_LAYERS + 1) * 8 + 1)
    new_cells = 0
    for l, o in zip((1, 2), old):
        nl = n0 * r ** l
        a_new = np.zeros((nl, nl), bool)
        a_old = np.zeros((nl, nl), bool)
        for (i0, j0, i1, j1) in H.get_patches(0, l).tolist():
            a_new[j0:j1, i0:i1] = True
        for (i0, j0, i1, j1) in o.tolist():
            a_old[j0:j1, i0:i1] = True
        new_cells += int((a_new & ~a_old).sum())
    ib = new_cells * (3 * M_LAYERS + 1) * 8
    transfers["regrid"] = {"wall_ms": regrid_s * 1e3, "flags_ms": per["flags"][0],
                           "flags_algorithmic_bytes": fb,
                           "flags_achieved_gbs": fb / (per["flags"][0] * 1e-3) / 1e9 if per["flags"][0] else None,
                           "interp_ms": per["interp_fine"][0], "new_fine_cells": new_cells,
                           "interp_algorithmic_bytes": ib,
                           "interp_achieved_gbs": ib / (per["interp_fine"][0] * 1e-3) / 1e9
                           if per["interp_fine"][0] else None,
                           "patches_after": [len(H.get_patches(0, l)) for l in (1, 2)]}
    # the whole AMR cycle: 8 coarse steps with a regrid before every 4th (as the workload's
    # regrid interval), cell updates from the device counters, regrids inside the timed region
    H.advance(1)
    torch.cuda.synchronize()
    s0 = H.get_stats()
    t0 = time.perf_counter()
    for _ in range(2):
        H.regrid(0)
        H.advance(4)
    torch.cuda.synchronize()
    cyc_s = time.perf_counter() - t0
    s1 = H.get_stats()
    cyc_upd = sum(s1["cell_updates"]) - sum(s0["cell_updates"])
    transfers["cycle_with_regrids"] = {"coarse_steps": 8, "regrids": 2, "wall_ms": cyc_s * 1e3,
                                       "cell_updates": cyc_upd, "lcups": cyc_upd * M_LAYERS / cyc_s,
                                       "patches": [len(H.get_patches(0, l)) for l in (1, 2)]}
    transfers["partition_exchange"] = _partition_pack_times(torch, H, stream)
    H.close()
    lb = upd * M_LAYERS * steps / (ms_b * 1e-3)
    lp = upd * M_LAYERS * max(1, steps // 2) / (ms_p * 1e-3)
    return {"workload": f"3 levels, {n0}^2 coarse, ratios 4,4, shore bathymetry, 8 humps; seeded layout of "
                        f"{n_patches[0]} level-1 and {n_patches[1]} level-2 patches (sides 16..64)",
            "cell_updates_per_coarse_step": upd, "coarse_steps": steps,
            "lcups_batched": lb, "lcups_per_patch": lp, "batched_over_per_patch": lb / lp,
            "ms_per_coarse_step_batched": ms_b / steps, "ms_per_coarse_step_per_patch": ms_p / max(1, steps // 2),
            "autotuned_tiles": chosen, "level_transfers": transfers}


def _partition_pack_times(torch, H, stream, ws=2, reps=5):
    """Kernel side of the patch-partition exchange on one GPU: the hierarchy split over ws
    ranks (no hook; this process plays rank 0), then per refined level the doubles every rank
    sends in a full exchange, the job's bytes of the other kinds of exchange (halo, last,
    averaged), and the pack and unpack times of rank 0's and rank 1's full buffers (CUDA
    events; read + write bytes of the copies over the time)."""
    H.set_partition(0, ws)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {"ranks": ws}
    for level in (1, 2):
        sizes = H.partition_sizes(level)
        buf = torch.empty(max(sizes), dtype=torch.float64, device=dev)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e[0].record(stream)
        for _ in range(reps):
            H.partition_pack(level, buf.data_ptr())
        e[1].record(stream)
        for _ in range(reps):
            H.partition_unpack(level, 1, buf.data_ptr())
        e[2].record(stream)
        torch.cuda.synchronize()
        pack_ms, unpack_ms = e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps
        kinds = {k: 8 * sum(H.partition_sizes(level, i)) for i, k in ((1, "halo"), (2, "last"))}
        if level == 1:
            kinds["averaged_into_level1"] = 8 * sum(H.partition_sizes(1, 3))
        out[f"level{level}"] = {"doubles_per_rank": sizes, "job_bytes_per_level_step": 8 * sum(sizes),
                                "job_bytes_of_other_kinds": kinds,
                                "pack_ms": pack_ms, "pack_gbs": 16 * sizes[0] / (pack_ms * 1e-3) / 1e9,
                                "unpack_ms": unpack_ms, "unpack_gbs": 16 * sizes[1] / (unpack_ms * 1e-3) / 1e9}
    H.set_partition(0, 1)
    return out


def bench_amr_partitioned(pkg, torch, stream, rank, ws, steps=3, n0=512, patches=(1000, 3000)):
    """The batched AMR workload with the patches of its refined levels split over the ranks
    (space-filling curve, balanced cells): every rank holds the whole hierarchy and sweeps its
    own patches; after each refined level step the ranks all-gather their packed patch values
    and take the largest wave speeds over NCCL (sharding.PatchPartition). Layer-cell updates of
    the job (every rank's hierarchy is the whole job) over the slowest rank's time."""
    import torch.distributed as dist
    from paper_1803_01450_gb300 import sharding as S
    H, _, upd = _batched_amr_hierarchy(pkg, stream, n0, patches)
    dev = torch.device("cuda", torch.cuda.current_device())
    S.PatchPartition(H, rank, ws, dist, dev)
    H.advance(1)
    torch.cuda.synchronize()
    dist.barrier()
    ms = _time_advance(torch, H, stream, steps)
    H.close()
    tmax = S.max_all(ms, dist, dev)
    return {"workload": f"3 levels, {n0}^2 coarse, {patches[0]} + {patches[1]} patches split over {ws} ranks",
            "ranks": ws, "lcups": upd * M_LAYERS * steps / (tmax * 1e-3),
            "ms_per_coarse_step_slowest_rank": tmax / steps}


def _batched_amr_hierarchy(pkg, stream, n0, patches, autotune=True):
    """The three-level hierarchy of the batched AMR workload (shore bathymetry, 8 humps, seeded
    synthetic layouts of patches[0] level-1 and patches[1] level-2 patches), its autotuned
    tiles and its interior cell updates per coarse step."""
    r = 4
    nf = n0 * r * r
    L = 1e5
    cfg = pkg.Config(M=2, dry_tol=1e-3, max_levels=3, ratio=[r, r], regrid_interval=0, min_side=16, max_side=64,
                     flag_tol=5e-5)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, L, L, n0, n0)], stream=stream.cuda_stream)
    xf = I.centers(0.0, L, nf)
    Bf = np.ascontiguousarray(np.broadcast_to(I.shore_B(xf)[None, :], (nf, nf)))
    H.set_bathymetry(0, Bf)
    del Bf
    B0 = H.get_bathymetry(0, 0)
    x0 = I.centers(0.0, L, n0)
    X, Y = np.meshgrid(x0, x0)
    eta1 = I.hump_field(X, Y, *I.humps(3000, 8))
    H.set_state(0, 0, I.layered_state(B0, eta1, -200.0 * np.ones_like(B0)))
    l1 = I.random_layout(3100, n0 * r, n0 * r, patches[0], r)
    l2 = I.random_layout(3200, nf, nf, patches[1], r, parents=l1, margin=2)
    H.set_patches(0, 1, l1)
    H.interp_fine(0, 0)
    H.set_patches(0, 2, l2)
    H.interp_fine(1, 0)
    chosen = [H.autotune(l, iters=2) for l in range(3)] if autotune else None
    return H, chosen, _interior_updates(H, 1, 3, [r, r])



def bench_dynamic_rt(pkg, torch, stream, steps=6):
    """Three levels refined on the coastal strip of the shore bathymetry (x in 86..99 km, 340 m
    deep at most against 4000 m offshore), advanced with the fixed time ratios and with the
    dynamic ones (fewest substeps that keep each level at the Courant target): simulated time
    per wall second, level steps and cell updates per coarse step for both."""
    n0, r = 512, 4
    nf = n0 * r * r
    L = 1e5
    xf = I.centers(0.0, L, nf)
    Bf = np.ascontiguousarray(np.broadcast_to(I.shore_B(xf)[None, :], (nf, nf)))
    x0 = I.centers(0.0, L, n0)
    X, Y = np.meshgrid(x0, x0)
    eta1 = I.hump_field(X, Y, *I.humps(3000, 8))
    strip = [(int(8.6e4 / L * n0), 0, int(9.9e4 / L * n0), n0)]  # coarse cells over the coastal strip
    l1 = I.random_layout(3300, n0 * r, n0 * r, 600, r, parents=strip, margin=2)
    l2 = I.random_layout(3400, nf, nf, 2000, r, parents=l1, margin=2)
    out = {"workload": "3 levels, 512^2 coarse, ratios 4,4, shore bathymetry, 8 humps; seeded layout of "
                       f"{len(l1)} level-1 and {len(l2)} level-2 patches on the coastal strip (x 86..99 km, 30..340 m deep)",
           "coarse_steps": steps}
    for dyn in (0, 1):
        cfg = pkg.Config(M=2, dry_tol=1e-3, max_levels=3, ratio=[r, r], regrid_interval=0, min_side=16,
                         max_side=64, dynamic_rt=dyn)
        H = pkg.Hierarchy(cfg, [(0.0, 0.0, L, L, n0, n0)], stream=stream.cuda_stream)
        H.set_bathymetry(0, Bf)
        B0 = H.get_bathymetry(0, 0)
        H.set_state(0, 0, I.layered_state(B0, eta1, -200.0 * np.ones_like(B0)))
        H.set_patches(0, 1, l1)
        H.interp_fine(0, 0)
        H.set_patches(0, 2, l2)
        H.interp_fine(1, 0)
        for l in range(3):
            H.autotune(l, iters=2)
        H.advance(1)
        s0 = H.get_stats()
        t0 = H.get_time()[0][0]
        ms = _time_advance(torch, H, stream, steps)
        s1 = H.get_stats()
        t1 = H.get_time()[0][0]
        H.close()
        upd = sum(s1["cell_updates"]) - sum(s0["cell_updates"])
        key = "dynamic" if dyn else "fixed"
        out[key] = {"ms_per_coarse_step": ms / steps, "sim_seconds_per_wall_second": (t1 - t0) / (ms * 1e-3),
                    "level_steps_per_coarse_step": [(b - a) / steps for a, b in
                                                    zip(s0["level_steps"], s1["level_steps"])],
                    "cell_updates_per_coarse_step": upd / steps,
                    "lcups": upd * M_LAYERS / (ms * 1e-3), "last_cfl": s1["last_cfl"]}
    out["dynamic_over_fixed_sim_rate"] = (out["dynamic"]["sim_seconds_per_wall_second"]
                                          / out["fixed"]["sim_seconds_per_wall_second"])
    return out


def _ensemble_hierarchy(pkg, stream, ids, r=4):
    """The ensemble workload's members `ids` (seeded shelves, humps and refined layouts) in one
    hierarchy, autotuned; returns (hierarchy, chosen tiles)."""
    members = [I.ensemble_member(k) for k in ids]
    cfg = pkg.Config(M=2, dry_tol=1e-3, max_levels=2, ratio=[r], regrid_interval=0, min_side=16, max_side=64)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, m["L"], m["L"], m["n"], m["n"]) for m in members], stream=stream.cuda_stream)
    for k, (mid, m) in enumerate(zip(ids, members)):
        nf = m["n"] * r
        xf = I.centers(0.0, m["L"], nf)
        Bf = np.ascontiguousarray(np.broadcast_to(I.shelf_B(xf, depth=m["depth"], shelf_x=m["shelf_x"])[None, :],
                                                  (nf, nf)))
        H.set_bathymetry(k, Bf)
        B0 = H.get_bathymetry(k, 0)
        x0 = I.centers(0.0, m["L"], m["n"])
        X, Y = np.meshgrid(x0, x0)
        H.set_state(k, 0, I.layered_state(B0, I.hump_field(X, Y, *m["humps"]), -200.0 * np.ones_like(B0)))
        H.set_patches(k, 1, I.random_layout(5100 + mid, m["n"] * r, m["n"] * r, max(4, m["n"] // 16), r))
        H.interp_fine(0, k)
    chosen = [H.autotune(l, iters=2) for l in range(2)]
    return H, chosen


def bench_ensemble_partitioned(pkg, torch, stream, rank, ws, n_members=256, steps=3):
    """The ensemble workload with its members partitioned over the ranks (largest first to the
    least-loaded rank, by level-0 cells); each rank advances its members in its own batched
    launches; the job's cell updates are summed and its time is the slowest rank's."""
    import torch.distributed as dist
    from paper_1803_01450_gb300 import sharding as S
    costs = [I.ensemble_member(k)["n"] ** 2 for k in range(n_members)]
    ids = S.partition_members(costs, ws)[rank]
    H, _ = _ensemble_hierarchy(pkg, stream, ids)
    upd = _interior_updates(H, len(ids), 2, [4])
    H.advance(1)
    torch.cuda.synchronize()
    dist.barrier()
    ms = _time_advance(torch, H, stream, steps)
    H.close()
    tmax = S.max_all(ms, dist, torch.device("cuda", torch.cuda.current_device()))
    total = S.sum_all(upd * M_LAYERS * steps, dist, torch.device("cuda", torch.cuda.current_device()))
    return {"workload": f"{n_members} ensemble members partitioned over {ws} ranks", "ranks": ws,
            "lcups": total / (tmax * 1e-3), "ms_slowest_rank": tmax, "members_per_rank": len(ids)}


def bench_slabs(pkg, torch, stream, rank, ws, n=N_CELLS, steps=10, warmup=3):
    """The headline grid split into slabs of rows over the ranks, two halo rows swapped by
    NCCL point-to-point sends before every step; owned layer-cell updates of all ranks over the
    slowest rank's time (strong scaling of one grid)."""
    import torch.distributed as dist
    from paper_1803_01450_gb300 import sharding as S
    w = I.scale(n, seed=1000)
    sl = S.slab_of(n, ws, rank)
    dy = 1e5 / n
    cfg = pkg.Config(M=2, dry_tol=w["dry_tol"], order=2, limiter=2, max_levels=1)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1e5, sl.rows * dy, n, sl.rows)], stream=stream.cuda_stream)
    H.set_bathymetry(0, np.ascontiguousarray(w["B"][sl.lo:sl.hi]))
    H.set_state(0, 0, np.ascontiguousarray(w["q"][:, sl.lo:sl.hi]))
    H.set_dt(0, 0.9 * w["dx"] / 205.0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def get_rows(r0, k):
        t = torch.empty((3 * M_LAYERS, k, n), dtype=torch.float64, device=dev)
        H.get_rows_device(0, 0, r0, k, t.data_ptr())
        return t

    def set_rows(r0, k, t):
        H.set_rows_device(0, 0, r0, k, t.data_ptr())

    def step():
        with torch.cuda.stream(stream):
            S.halo_exchange(sl, rank, ws, get_rows, set_rows, dist)
        H.step_level(0)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    H.close()
    tmax = S.max_all(ms, dist, dev)
    total = S.sum_all((sl.j1 - sl.j0) * n * M_LAYERS * steps, dist, dev)
    return {"workload": f"{n}x{n} shelf grid in {ws} slabs of rows, 2 halo rows per shared edge", "ranks": ws,
            "lcups": total / (tmax * 1e-3), "ms_per_step_slowest_rank": tmax / steps}


def bench_ensemble(pkg, torch, stream, n_members=256, steps=3):
    """Ensemble of independent members, U{128..512}^2 coarse grids, one refined level."""
    r = 4
    H, chosen = _ensemble_hierarchy(pkg, stream, list(range(n_members)), r)
    upd = _interior_updates(H, n_members, 2, [r])
    H.advance(1)
    ms_b = _time_advance(torch, H, stream, steps)
    H.set_execution(use_graphs=False, per_patch_launches=True)
    H.advance(1)
    ms_p = _time_advance(torch, H, stream, steps)
    t, dt = H.get_time()
    dev_gb = torch.cuda.max_memory_allocated() / 1e9
    H.close()
    lb = upd * M_LAYERS * steps / (ms_b * 1e-3)
    lp = upd * M_LAYERS * steps / (ms_p * 1e-3)
    return {"workload": f"{n_members} members, coarse U{{128..512}}^2, seeded shelf depth/position and 1-4 humps, "
                        "1 refined level (ratio 4, seeded patches)",
            "members": n_members, "cell_updates_per_coarse_step": upd, "coarse_steps": steps,
            "lcups_batched": lb, "lcups_per_patch": lp, "batched_over_per_patch": lb / lp,
            "distinct_member_dt": int(len(set(np.round(dt, 12)))), "autotuned_tiles": chosen,
            "peak_device_gb": dev_gb}


def bench_adjoint_forms(pkg, torch, stream):
    """The adjoint workload with checkpoints every 20 steps (the figure), and as one segment
    whose per-edge forward records all stay in HBM (no recomputation in the backward pass)."""
    out = bench_adjoint(pkg, torch, stream)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    one = bench_adjoint(pkg, torch, stream, ckpt=200)
    out["single_segment"] = {"checkpoint_every": 200, "forward_ms": one["forward_ms"],
                             "backward_ms": one["backward_ms"], "adjoint_over_forward": one["adjoint_over_forward"],
                             "peak_device_gb": torch.cuda.max_memory_allocated() / 1e9}
    return out


def bench_adjoint(pkg, torch, stream, n=512, steps=200, ckpt=20, n_g=32):
    """Gauge-misfit gradient on the 512^2 adjoint workload: forward (200 first-order steps,
    loss) versus backward (segment recomputation from checkpoints + transposed steps)."""
    from paper_1803_01450_gb300.adjoint import FixedGridProblem
    L = 1e5
    B = I.adjoint_bathymetry(n, L)
    eta1 = I.adjoint_eta1(n, seed=4000, L=L)
    gauges = I.gauge_cells(n, n_g, seed=4100)
    dt = 0.5 * (L / n) / 205.0
    obs = np.zeros((steps, n_g))  # the cost does not depend on the observed values
    prob = FixedGridProblem(n, n, L, dt, steps, ckpt, gauges, obs, stream=stream.cuda_stream)
    dev = torch.device("cuda", torch.cuda.current_device())
    eta1_d = torch.as_tensor(eta1, dtype=torch.float64, device=dev)
    B_d = torch.as_tensor(B, dtype=torch.float64, device=dev)
    prob.forward(eta1_d, B_d, dev)  # setup (tile timing) and a first pass
    prob.control_gradient(dev)
    d_eta1 = torch.empty((n, n), dtype=torch.float64, device=dev)
    d_B = torch.empty((n, n), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    # the timed calls are the C ABI's: controls -> loss, then loss -> control gradients
    e[0].record(stream)
    loss = prob.H.fixed_forward(eta1_d.data_ptr(), B_d.data_ptr(), prob.eta2)
    e[1].record(stream)
    torch.cuda.synchronize()
    e[1].synchronize()
    t_b0 = torch.cuda.Event(enable_timing=True)
    t_b0.record(stream)
    prob.H.fixed_backward(d_eta1.data_ptr(), d_B.data_ptr())
    e[2].record(stream)
    torch.cuda.synchronize()
    fwd = e[0].elapsed_time(e[1])
    bwd = t_b0.elapsed_time(e[2])
    prob.close()
    return {"workload": f"{n}^2 fixed grid, 2 layers, B = -4000 + 500 sin cos, 8 humps, order 1, fixed dt, "
                        f"{steps} steps, {n_g} gauges, checkpoint every {ckpt}",
            "forward_ms": fwd, "backward_ms": bwd, "adjoint_over_forward": bwd / fwd,
            "forward_lcups": n * n * M_LAYERS * steps / (fwd * 1e-3), "loss": loss}


def bench_three_layers(pkg, torch, stream, n=N_CELLS, steps=10, warmup=3, M=3):
    """The headline workload with three layers (surfaces humps / -100 m / -600 m over the same
    shelf, densities 1000 / 1020 / 1030), or four (humps / -100 / -300 / -600 m, densities
    1000 / 1020 / 1030 / 1040): the general M-layer coupled branch in deep water, the
    per-layer branch on the shelf where the lower layers end."""
    w = I.scale3(n, seed=1000) if M == 3 else I.scale4(n, seed=1000)
    rho = (1000.0, 1020.0, 1030.0, 1040.0)[:M]
    flop = FP64_FLOP_PER_CELL_UPDATE_3 if M == 3 else FP64_FLOP_PER_CELL_UPDATE_4
    cfg = pkg.Config(M=M, rho=rho, dry_tol=w["dry_tol"], order=2, limiter=2, max_levels=1)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1e5, 1e5, n, n)], stream=stream.cuda_stream)
    H.set_bathymetry(0, w["B"])
    H.set_state(0, 0, w["q"])
    tiles = H.autotune(0, iters=2)
    H.set_dt(0, 0.9 * w["dx"] / 205.0)
    for _ in range(warmup):
        H.step_level(0)
    torch.cuda.synchronize()
    H.timing(enable=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        H.step_level(0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    per_kernel, _ = H.timing(enable=False)
    H.close()
    sx_ms, sx_n = per_kernel["sweep_x"]
    x_ms = sx_ms / max(1, sx_n)
    ach = 0.5 * flop * n * n / (x_ms * 1e-3) / 1e12
    surf = "-100 m / -600 m" if M == 3 else "-100 m / -300 m / -600 m"
    return {"workload": f"{n}^2 shelf, {M} layers (humps / {surf}), order 2 MC, walls",
            "lcups": n * n * M * steps / (ms * 1e-3), "ms_per_step": ms / steps, "sweep_x_ms": x_ms,
            "flop_per_cell_update": flop, "achieved_tflops": ach,
            "frac_of_fp64_peak": ach / FP64_PEAK_TFLOPS, "tiles": tiles}


def bench_unsplit(pkg, torch, stream, n=N_CELLS, steps=10, warmup=3):
    """The headline workload with the unsplit step (transverse Riemann solves): throughput,
    the x edge pass against the FP64 peak, and the update kernel against HBM (it reads the
    12 x 3M per-edge values, the state, and writes the state: 14 x 3M doubles per cell)."""
    w = I.scale(n, seed=1000)
    cfg = pkg.Config(M=2, dry_tol=w["dry_tol"], order=2, limiter=2, max_levels=1, unsplit=1)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1e5, 1e5, n, n)], stream=stream.cuda_stream)
    H.set_bathymetry(0, w["B"])
    H.set_state(0, 0, w["q"])
    tiles = H.autotune(0, iters=2)
    H.set_dt(0, 0.9 * w["dx"] / 205.0)
    for _ in range(warmup):
        H.step_level(0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        H.step_level(0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    H.timing(enable=True)
    for _ in range(steps):
        H.step_level(0)
    torch.cuda.synchronize()
    per_kernel, _ = H.timing(enable=False)
    H.close()
    kms = {k: v[0] / v[1] for k, v in per_kernel.items() if v[1]}
    x_ms = kms["sweep_x"]
    ach = FP64_FLOP_UNSPLIT_EDGE_PASS * n * n / (x_ms * 1e-3) / 1e12
    upd_bytes = 14 * 3 * M_LAYERS * 8 * n * n
    upd_gbs = upd_bytes / (kms["update"] * 1e-3) / 1e9
    # three layers (the scale3 workload) with the unsplit step
    w3 = I.scale3(n, seed=1000)
    cfg3 = pkg.Config(M=3, rho=(1000.0, 1020.0, 1030.0), dry_tol=w3["dry_tol"], order=2, limiter=2, max_levels=1,
                      unsplit=1)
    H3 = pkg.Hierarchy(cfg3, [(0.0, 0.0, 1e5, 1e5, n, n)], stream=stream.cuda_stream)
    H3.set_bathymetry(0, w3["B"])
    H3.set_state(0, 0, w3["q"])
    H3.set_dt(0, 0.9 * w3["dx"] / 205.0)
    for _ in range(warmup):
        H3.step_level(0)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        H3.step_level(0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms3 = e0.elapsed_time(e1)
    H3.close()
    return {"workload": f"{n}^2 shelf, 2 layers, 8 humps, order 2 MC, walls, unsplit step",
            "three_layers_lcups": n * n * 3 * steps / (ms3 * 1e-3), "three_layers_ms_per_step": ms3 / steps,
            "three_layers_step_tflops": FP64_FLOP_PER_CELL_UPDATE_UNSPLIT_3 * n * n / (ms3 / steps * 1e-3) / 1e12,
            "lcups": n * n * M_LAYERS * steps / (ms * 1e-3), "ms_per_step": ms / steps,
            "kernels_ms_per_launch": kms, "flop_per_cell_update": FP64_FLOP_PER_CELL_UPDATE_UNSPLIT,
            "x_pass_achieved_tflops": ach, "x_pass_frac_of_fp64_peak": ach / FP64_PEAK_TFLOPS,
            "update_achieved_gbs": upd_gbs, "update_frac_of_hbm": upd_gbs / HBM_PEAK_GBS,
            "update_algorithmic_bytes": upd_bytes, "tiles": tiles}


def _summary(line):
    """The secondary figures in a few numbers, last on the line (readers that keep only the
    end of the output still see them)."""
    out = {"headline_lcups": line["value"], "e2e_lcups": line["e2e"]["value"],
           "sweep_frac_of_fp64_peak": line["roofline"]["frac"]}
    amr = line.get("batched_amr")
    if amr:
        out["batched_amr"] = {"batched_lcups": amr.get("lcups_batched"), "per_patch_lcups": amr.get("lcups_per_patch"),
                              "ratio": amr.get("batched_over_per_patch")}
    ens = line.get("ensemble")
    if ens:
        out["ensemble"] = {"batched_lcups": ens.get("lcups_batched"), "per_patch_lcups": ens.get("lcups_per_patch"),
                           "ratio": ens.get("batched_over_per_patch")}
    adj = line.get("adjoint")
    if adj:
        out["adjoint_over_forward"] = adj.get("adjoint_over_forward")
    for key in ("ensemble_partitioned", "slabs", "amr_partitioned"):
        if key in line:
            out[key + "_lcups"] = line[key]["lcups"]
    cpu = line.get("cpu_baseline")
    if cpu:
        out["cpu_oracle_lcups"] = cpu["value"]
        out["cpu_oracle_one_core_lcups"] = (cpu.get("one_core") or {}).get("value")
    return out


def run_only(name, args=None):
    import functools
    import torch
    import paper_1803_01450_gb300 as pkg
    pkg.build()
    stream = torch.cuda.Stream()
    amr = bench_batched_amr
    if args is not None and args.amr_coarse:
        a, b = (int(v) for v in args.amr_patches.split(","))
        amr = functools.partial(bench_batched_amr, n0=args.amr_coarse, patches=(a, b))
    fn = {"amr": amr, "ensemble": bench_ensemble, "adjoint": bench_adjoint_forms,
          "three": bench_three_layers, "four": functools.partial(bench_three_layers, M=4), "dynrt": bench_dynamic_rt, "unsplit": bench_unsplit}[name]
    key = {"amr": "batched_amr", "ensemble": "ensemble", "adjoint": "adjoint", "three": "three_layers",
           "four": "four_layers",
           "dynrt": "dynamic_time_ratio", "unsplit": "unsplit"}[name]
    print(json.dumps({key: fn(pkg, torch, stream)}), flush=True)


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

    # Each rank advances its own replica of the headline workload (independent problems).
    w = I.scale(N_CELLS, seed=replica_seed(rank))
    cfg = pkg.Config(M=2, dry_tol=w["dry_tol"], order=2, limiter=2, max_levels=1)
    stream = torch.cuda.Stream(device=dev)
    H = pkg.Hierarchy(cfg, [(0.0, 0.0, 1e5, 1e5, N_CELLS, N_CELLS)], stream=stream.cuda_stream)
    H.set_bathymetry(0, w["B"])
    H.set_state(0, 0, w["q"])
    tiles = "default 125 x 2, 2 CTAs per SM" if args.no_autotune else H.autotune(0, iters=3)
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

    # ---- end to end through the public API with pinned host buffers ----
    # Every step copies its input state from pinned host memory and reads its gauges back.
    # Pipelined: the input of step k + 1 is enqueued (copy stream, double-buffered staging)
    # right after step k, so its host-to-device copy overlaps step k's compute, and the host
    # waits for step k - 1's gauges (an event on the stream) while step k runs.
    # the input every step uploads: the state the device-timed steps reached (the same flow,
    # so both regions do the same work per step)
    qh = torch.empty(w["q"].shape, dtype=torch.float64, pin_memory=True).numpy()
    qh[...] = H.get_state(0, 0)
    xy = np.stack([np.linspace(1e4, 9e4, 32), np.linspace(2e4, 8e4, 32)], axis=1)
    gout = [torch.empty((32, M_LAYERS), dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    results = []
    e2e_steps = max(3, args.steps)  # the timed region's K steps (the first input copy is not overlapped)
    H.set_state(0, 0, qh)
    H.step_level(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H.set_state_async(0, 0, qh)
    for k in range(e2e_steps):
        H.step_level(0)
        H.read_gauges_async(0, xy, gout[k % 2])
        done[k % 2].record(stream)
        if k + 1 < e2e_steps:
            H.set_state_async(0, 0, qh)
        if k >= 1:
            done[(k - 1) % 2].synchronize()
            results.append(gout[(k - 1) % 2].copy())
    done[(e2e_steps - 1) % 2].synchronize()
    results.append(gout[(e2e_steps - 1) % 2].copy())
    H.synchronize()
    e2e_s = time.perf_counter() - t0
    assert len(results) == e2e_steps and all(np.isfinite(g).all() for g in results)
    H.close()

    lcu_per_step = N_CELLS * N_CELLS * M_LAYERS
    tmax = max_over_ranks(ms, ws, dev)
    value = job_value(lcu_per_step, args.steps, ws, tmax)
    e2e_value = job_value(lcu_per_step, e2e_steps, ws, max_over_ranks(e2e_s * 1e3, ws, dev))

    sx_ms, sx_n = per_kernel["sweep_x"]
    sy_ms, sy_n = per_kernel["sweep_y"]
    x_launch_ms = sx_ms / max(1, sx_n)
    ach = 0.5 * FP64_FLOP_PER_CELL_UPDATE * N_CELLS * N_CELLS / (x_launch_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": "sweep_kernel<2,0> (x sweep)", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": SWEEP_X_DRAM_BYTES,
            "flop_per_launch": 0.5 * FP64_FLOP_PER_CELL_UPDATE * N_CELLS * N_CELLS,
            "launch_ms": x_launch_ms, "y_sweep_launch_ms": sy_ms / max(1, sy_n),
            "peak_note": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz; a DFMA-chain microbenchmark "
                         "reaches 1.012 TFLOP/s on this part"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_name(), "cells": N_CELLS * N_CELLS, "layers": M_LAYERS,
                   "l2": "inputs larger than L2 (201 MB state per buffer), no flush",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU", "tiles": tiles},
        "clocks": clocks,
        "gpu_launches": total_launches,
        "kernels_ms_per_launch": {k: (v[0] / v[1] if v[1] else None) for k, v in per_kernel.items() if v[1]},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(w["q"].nbytes + xy.nbytes) * ws, "d2h_bytes_per_step": 32 * M_LAYERS * 8 * ws},
    }
    if ws > 1 and not args.no_amr:
        # work split over the ranks (every rank takes part): members partitioned, one grid in slabs
        part = bench_ensemble_partitioned(pkg, torch, stream, rank, ws)
        slabs = bench_slabs(pkg, torch, stream, rank, ws)
        amr_part = bench_amr_partitioned(pkg, torch, stream, rank, ws)
        if rank == 0:
            line["ensemble_partitioned"] = part
            line["slabs"] = slabs
            line["amr_partitioned"] = amr_part
    if rank == 0 and ws == 1 and not args.no_amr:
        # single-GPU figures (with N > 1 GPUs they would hold every GPU while rank 0 repeats
        # the N = 1 run's numbers)
        line["batched_amr"] = bench_batched_amr(pkg, torch, stream)
        line["ensemble"] = bench_ensemble(pkg, torch, stream)
        line["adjoint"] = bench_adjoint_forms(pkg, torch, stream)
        line["three_layers"] = bench_three_layers(pkg, torch, stream)
        line["four_layers"] = bench_three_layers(pkg, torch, stream, M=4)
        line["dynamic_time_ratio"] = bench_dynamic_rt(pkg, torch, stream)
        line["unsplit"] = bench_unsplit(pkg, torch, stream)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        line["summary"] = _summary(line)
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
    ap.add_argument("--no-amr", action="store_true", help="skip the batched-AMR, ensemble and adjoint figures")
    ap.add_argument("--no-autotune", action="store_true",
                    help="headline sweeps with the default tiles (no tile trials before the timed steps)")
    ap.add_argument("--amr-coarse", type=int, default=0,
                    help="with --only amr: coarse grid side of a smaller case (default: the 512 figure)")
    ap.add_argument("--amr-patches", default="1000,3000", help="with --amr-coarse: level-1,level-2 patch counts")
    ap.add_argument("--only", choices=["amr", "ensemble", "adjoint", "three", "four", "dynrt", "unsplit"],
                    help="print only that secondary figure (a short command for profiling its kernels)")
    args = ap.parse_args()
    if args.only:
        run_only(args.only, args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
