#!/usr/bin/env python
"""Throughput of the coupled free-surface LBM / DEM time step on GB300.

One bench step is one full time step of the method (stream-collide with all
boundary conditions and momentum exchange, free-surface update, DEM
sub-steps, particle re-mapping) on the 3072x96x320 flume workload (~94 M
cells, seeded particle bed). Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (one process per GPU under torch.distributed.run) every rank runs
an independent replica with its own seed: the method has no exchange step at
this size, so there is no data-path collective; the barrier and the
max-over-ranks timing use the process group.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = None
UNIT = "MLUPS"
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
ELEM = {"fp32": 4, "fp16": 2, "bf16": 2}


def _metric_name() -> str:
    try:
        with open(os.path.join(ROOT, "BASELINE.json")) as f:
            return json.load(f)["metric"]
    except Exception:
        return "coupled FSLBM-DEM MLUPS"


def _peaks() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _workload(name: str, rank: int):
    from paper_2301_10674_gb300 import workloads as W
    w = W.WORKLOADS[name]()
    w.seed += 1000 * rank
    return w.generate()


# ---------------------------------------------------------------- oracle leg

def run_oracle(w, steps: int, warmup: int, crop_nx: int) -> dict:
    """The FP64 oracle on an x-crop of the same workload (host cores)."""
    import oracle as O
    c = w.crop_x(crop_nx)
    o = O.Oracle(O.OracleParams(
        nx=c.nx, ny=c.ny, nz=c.nz, periodic=tuple(c.periodic), omega=c.omega, g=tuple(c.g), rho_gas=c.rho_gas,
        liquid_height=c.liquid_height, eps_conv=c.eps_conv, eps_normal=c.eps_normal,
        reconstruct_normal=c.reconstruct_normal, rho_p=c.rho_p, restitution=c.restitution, friction=c.friction,
        poisson=c.poisson, collision_time=c.collision_time, dem_substeps=c.dem_substeps))
    if c.nspheres:
        o.add_spheres(c.xyz, c.radius, c.fixed)
    o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cells = c.nx * c.ny * c.nz
    return {"value": cells * steps / dt / 1e6, "cores": O.threads(), "seconds": dt,
            "sample": f"{c.nx}x{c.ny}x{c.nz} x-crop of {w.name} ({c.nspheres} spheres), {steps} steps "
                      f"after {warmup} warm-up steps"}


# ---------------------------------------------------------------- GPU leg

def run_ours(args, world, rank, local):
    import torch

    from paper_2301_10674_gb300 import build as B
    from paper_2301_10674_gb300 import fslbm as F

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    w = _workload(args.workload, rank)
    storage = STORAGE[args.storage]
    stream = torch.cuda.Stream()
    sim = F.Simulation.from_workload(w, storage=storage, stream=stream)
    ncell = w.ncells

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    sim.step(args.warmup)
    sim.sync()
    counts = sim.cell_counts()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    sim.timing(True)
    t_start.record(stream)
    sim.step(args.steps)
    t_end.record(stream)
    t_end.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = t_start.elapsed_time(t_end)
    sweep_ms, sweeps, launches = sim.timing_read()
    sim.timing(False)
    clk = clocks.stop()
    counts_after = sim.cell_counts()
    violations = sim.violations
    red = sim.reduce()
    sim.close()
    del sim

    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    else:
        ms_max = ms
    value = world * ncell * args.steps / (ms_max / 1e3) / 1e6

    # roofline of the stream-collide sweep: algorithmic bytes per launch
    elem = ELEM[args.storage]
    fluid = int(counts[1] + counts[2] + counts_after[1] + counts_after[2]) / 2.0
    other = ncell - fluid
    bytes_per_sweep = fluid * (54 * elem + 1) + other * 1
    sweep_s = sweep_ms / 1e3 / max(1, sweeps)
    achieved = bytes_per_sweep / sweep_s / 1e9
    peak, peak_kind = _peaks()

    # end to end through the public API with host buffers: create, add the
    # particle bed from pinned host memory, step, read the diagnostics back
    # every step, destroy
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, w, storage, stream, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_oracle(w, steps=args.cpu_steps, warmup=1, crop_nx=args.cpu_crop)
        cpu = {"value": cpu["value"], "unit": UNIT, "cores": cpu["cores"], "kind": "oracle", "sample": cpu["sample"]}

    if rank != 0:
        return None
    out = {
        "metric": _metric_name(), "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "lattice": [w.nx, w.ny, w.nz], "cells": ncell,
                   "spheres": w.nspheres, "spheres_nominal": w.spheres_nominal, "storage": args.storage,
                   "cells_by_type": {"gas": int(counts_after[0]), "liquid": int(counts_after[1]),
                                     "interface": int(counts_after[2]), "solid": int(counts_after[3])},
                   "l2": f"no flush: the PDF lattice ({27 * 2 * elem * ncell / 1e9:.1f} GB incl. side buffer) "
                         f"is far larger than L2", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": "stream-collide sweep (bulk + boundary kernels)",
                     "bytes_per_launch": int(bytes_per_sweep), "launch_ms": round(sweep_s * 1e3, 4),
                     "peak_kind": peak_kind},
        "clocks": clk,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "checks": {"invariant_violations": int(violations), "liquid_mass": float(red[0]),
                   "interface_cells": int(red[5])},
    }
    return out


def run_e2e(args, w, storage, stream, world):
    import torch

    from paper_2301_10674_gb300 import fslbm as F

    xyz = torch.from_numpy(np.ascontiguousarray(w.xyz)).pin_memory().numpy()
    rad = torch.from_numpy(np.ascontiguousarray(w.radius)).pin_memory().numpy()
    fix = torch.from_numpy(np.ascontiguousarray(w.fixed)).pin_memory().numpy()
    diag = torch.empty(8, dtype=torch.float64).pin_memory().numpy()
    params = F.params_from_workload(w, storage)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = F.fslbm_create(params, stream.cuda_stream)
    F._check(F.fslbm_add_spheres(h, xyz, rad, fix), "fslbm_add_spheres")
    for _ in range(args.steps):
        F._check(F.fslbm_step(h, 1), "fslbm_step")
        rc, out = F.fslbm_reduce(h)
        F._check(rc, "fslbm_reduce")
        diag[:] = out
    F.fslbm_destroy(h)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([dt], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = float(t.item())
    h2d = xyz.nbytes + rad.nbytes + fix.nbytes + __import__("ctypes").sizeof(params)
    return {"value": round(world * w.ncells * args.steps / dt / 1e6, 2), "unit": UNIT,
            "h2d_bytes_per_step": round(h2d / args.steps, 1), "d2h_bytes_per_step": 64,
            "seconds": round(dt, 3),
            "note": "create + particle bed from pinned host memory + per step (fslbm_step, fslbm_reduce "
                    "read back to host) + destroy"}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    w = _workload(args.workload, 0)
    r = run_oracle(w, steps=args.steps, warmup=args.warmup, crop_nx=args.ref_crop)
    line = {
        "impl": "reference", "metric": _metric_name(), "value": round(r["value"], 4), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(r["seconds"] / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "lattice": [w.nx, w.ny, w.nz], "cells": w.ncells,
                   "sample_lattice": [args.ref_crop, w.ny, w.nz], "parallelism": "host cores"},
        "cpu_baseline": {"value": round(r["value"], 4), "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                         "sample": r["sample"]},
        "e2e": {"value": round(r["value"], 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="large")
    ap.add_argument("--storage", choices=tuple(STORAGE), default="fp32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--cpu-crop", type=int, default=64)
    ap.add_argument("--ref-crop", type=int, default=4)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = _dist()
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    else:
        line = run_ours(args, world, rank, local)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
