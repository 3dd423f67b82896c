#!/usr/bin/env python
"""Throughput of the coupled free-surface LBM / DEM time step on GB300.

One bench step is one full time step of the method (stream-collide with all
boundary conditions and momentum exchange, free-surface update, DEM
sub-steps, particle re-mapping) on the 3072x96x320 flume workload (~94 M
cells, seeded particle bed). Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--storage fp16|bf16|fp32] [--normals mlp|fd] [--no-compare]

The headline form stores the PDFs in FP16 (as f - w) and takes the interface
normal from the learned model, trained first (untimed) by the library's own
kernels on 4 M voxelised surfaces. The same steps are then timed for plain
FP32 with the finite-difference normal from the same initial state; the line
reports both, the speedup, and the difference between the two runs (mass
drift of each, liquid volume per column, bulk velocity).

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

UNIT = "MLUPS"
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
LINK_MODE = 0   # where the particle links are taken (--links: 0 the library's choice, 1 solid side, 2 fluid side)
MLP_MIRROR = True   # learned normal averaged over the mirror images in x and y (--no-mlp-mirror: the plain network)
ELEM = {"fp32": 4, "fp16": 2, "bf16": 2}


def _metric_name() -> str:
    return "coupled FSLBM-DEM MLUPS & %HBM roofline; FP16-store+MLP vs FP32 at stated error"


def _peaks() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _bf16_peak() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


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


def _max_over_ranks(x: float, device: str) -> float:
    """The largest value over the ranks of the process group (x alone
    without one): the timing of a multi-rank run is its slowest rank's."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _throughput(world: int, ncell: int, steps: int, seconds: float) -> float:
    """Whole-job MLUPS: every rank updates its own lattice of ncell cells."""
    return world * ncell * steps / seconds / 1e6


def _workload(name: str, rank: int):
    from paper_2301_10674_gb300 import workloads as W
    w = W.WORKLOADS[name]()
    w.seed += 1000 * rank
    return w.generate()


# ---------------------------------------------------------------- oracle leg

def run_oracle(w, steps: int, warmup: int, crop_nx: int, theta=None) -> dict:
    """The FP64 oracle on an x-crop of the same workload (host cores), with
    the learned normal when weights are given (rounded to BF16 as the GPU
    holds them)."""
    import oracle as O
    c = w.crop_x(crop_nx)
    o = O.Oracle(O.OracleParams(
        nx=c.nx, ny=c.ny, nz=c.nz, periodic=tuple(c.periodic), omega=c.omega, g=tuple(c.g), rho_gas=c.rho_gas,
        liquid_height=c.liquid_height, eps_conv=c.eps_conv, eps_normal=c.eps_normal,
        reconstruct_normal=c.reconstruct_normal, rho_p=c.rho_p, restitution=c.restitution, friction=c.friction,
        poisson=c.poisson, collision_time=c.collision_time, dem_substeps=c.dem_substeps))
    if c.nspheres:
        o.add_spheres(c.xyz, c.radius, c.fixed)
    if theta is not None:
        from paper_2301_10674_gb300 import fslbm as F
        bits = F.bf16_bits(theta).astype(np.uint32) << 16
        o.set_mlp(bits.view(np.float32).astype(np.float64), bf16=True, mirror=MLP_MIRROR)
    o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cells = c.nx * c.ny * c.nz
    return {"value": cells * steps / dt / 1e6, "cores": O.threads(), "seconds": dt,
            "sample": f"{c.nx}x{c.ny}x{c.nz} x-crop of {w.name} ({c.nspheres} spheres), {steps} steps "
                      f"after {warmup} warm-up steps"
                      + (", learned normal" if theta is not None else ", finite-difference normal")}


# ---------------------------------------------------------------- GPU leg

LAM, MU = 0.4, 0.1

# forms timed beside the headline one (storage, normal): plain FP32 with the
# finite-difference normal is the reference form of the comparison
COMPARE_FORMS = (("fp32", "fd"), ("fp16", "fd"), ("bf16", "fd"), ("fp32", "mlp"), ("fp16", "mlp"))

# DRAM traffic of the stream-collide sweep per fluid cell: dram__bytes_read.sum +
# dram__bytes_write.sum of every sweep kernel (links, liquid, rows, interface),
# even and odd steps averaged, from one ncu capture on the 1024x64x128 flume.
# It is valid while the sweep's sources hash to `sources`, and is scaled to a
# run by its fluid cells.
SWEEP_TRAFFIC = {"sources": "5e43e46c80f2ef71", "workload": "precision-1024x64x128",
                 "per_fluid_cell": {"fp16": 195.0, "fp32": 380.9, "bf16": 195.2}}
SWEEP_SOURCES = ("paper_2301_10674_gb300/csrc/stream_collide.cu", "paper_2301_10674_gb300/csrc/fslbm_dev.cuh",
                 "paper_2301_10674_gb300/csrc/collide_pair.cuh")


def _sweep_traffic(storage_name: str, fluid: float):
    import hashlib
    h = hashlib.sha256()
    for rel in SWEEP_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    per = SWEEP_TRAFFIC["per_fluid_cell"].get(storage_name)
    if per is None or h.hexdigest()[:16] != SWEEP_TRAFFIC["sources"]:
        return None, "no ncu capture of the current sweep for this storage"
    return int(per * fluid), (f"{per} B per fluid cell from an ncu capture on {SWEEP_TRAFFIC['workload']}, "
                              f"scaled by fluid cells")


def log_flume_stencils(stream, steps: int = 300, every: int = 50):
    """Interface stencils logged from a run of the mid flume (512x40x96, its
    particle bed, FP32, finite-difference normal) whose free surface starts
    with a seeded perturbation (amplitude 3 cells, x-wavelength 128, a
    y-modulation), labelled by the library's height function: every `every`
    steps, the snapshots alternating between training and held-out sets."""
    import torch

    from paper_2301_10674_gb300 import fslbm as F
    from paper_2301_10674_gb300 import workloads as W

    w = W.mid().generate()
    sim = F.Simulation.from_workload(w, storage=F.STORE_FP32, stream=stream)
    x = np.arange(w.nx) + 0.5
    y = np.arange(w.ny) + 0.5
    h = (w.liquid_height + 3.0 * np.sin(2 * np.pi * x / 128.0)[None, :] *
         (1.0 + 0.3 * np.cos(2 * np.pi * y / w.ny))[:, None])
    sim.init_surface(h)
    parts = ([], [])
    k = 0
    while k < steps:
        sim.step(every)
        k += every
        fill, target, fd, _ = sim.log_stencils()
        parts[(k // every) % 2].append((fill, target, fd))
    sim.close()
    cat = lambda ps, i: torch.cat([p[i] for p in ps]) if ps else None  # noqa: E731
    train = (cat(parts[0], 0), cat(parts[0], 1))
    held = (cat(parts[1], 0), cat(parts[1], 1), cat(parts[1], 2))
    return w.name, train, held


def _angles(a, b):
    a = a / np.linalg.norm(a, axis=1, keepdims=True)
    b = b / np.linalg.norm(b, axis=1, keepdims=True)
    return np.degrees(np.arccos(np.clip(np.sum(a * b, axis=1), -1.0, 1.0)))


def train_normal_model(stream, n_stencils: int, steps: int, seed: int = 4,
                       log_steps: int = 300) -> tuple[np.ndarray, dict]:
    """Learned normal trained by the library's own kernels (not timed):
    voxelised analytic surfaces (planes, droplets, bubbles, sine waves) and
    the stencils logged from a mid-flume run with their height-function
    labels, Adam on batches of 4096 with cube-symmetry augmentation, step
    size decaying geometrically from 2e-3 to 1e-5. The held-out logged
    stencils measure the network against the finite-difference normal on the
    method's own surfaces."""
    import torch

    from paper_2301_10674_gb300 import fslbm as F
    from paper_2301_10674_gb300 import workloads as W

    t0 = time.perf_counter()
    params = torch.from_numpy(W.surface_stencils(n_stencils, seed=seed)).cuda()
    fill = torch.empty((n_stencils, 27), dtype=torch.float32, device="cuda")
    tgt = torch.empty((n_stencils, 4), dtype=torch.float32, device="cuda")
    F._check(F.fslbm_mlp_stencils(params, n_stencils, fill, tgt, stream.cuda_stream), "fslbm_mlp_stencils")
    del params
    logged = None
    if log_steps > 0:
        log_name, (lf, lt), (hf, ht, hfd) = log_flume_stencils(stream, steps=log_steps)
        n_logged = len(lf)
        fill = torch.cat([fill, lf])
        tgt = torch.cat([tgt, lt])
        n_stencils = len(fill)
    t1 = time.perf_counter()
    theta = torch.from_numpy(W.mlp_initial_weights(seed)).cuda()
    curve = torch.empty(steps, dtype=torch.float32, device="cuda")
    F._check(F.fslbm_mlp_train(theta, fill, tgt, n_stencils, steps, 4096, 2e-3, LAM, MU, seed, True, curve,
                               stream.cuda_stream, lr_end=1e-5), "fslbm_mlp_train")
    t2 = time.perf_counter()
    c = curve.cpu().numpy()
    # the held-out logged stencils: the network with the step's fallback
    # rules (raw length in [1/2, 2], within 30 degrees of the
    # finite-difference normal) and the finite-difference normal, both
    # against the height-function labels
    if log_steps > 0:
        out = torch.empty((len(hf), 4), dtype=torch.float32, device="cuda")
        F._check(F.fslbm_mlp_infer(theta, hf, len(hf), out, stream.cuda_stream), "fslbm_mlp_infer")
        if MLP_MIRROR:
            # the network as the step uses it: averaged over the stencils'
            # mirror images in x, y and both, each output mapped back
            acc = out.clone()
            q = np.arange(27)
            for m in (1, 2, 3):
                a = 2 - q % 3 if m & 1 else q % 3
                b = 2 - (q // 3) % 3 if m & 2 else (q // 3) % 3
                idx = torch.from_numpy(a + 3 * b + 9 * (q // 9)).cuda()
                hm = hf[:, idx].contiguous()
                F._check(F.fslbm_mlp_infer(theta, hm, len(hf), out, stream.cuda_stream), "fslbm_mlp_infer")
                sign = torch.tensor([-1.0 if m & 1 else 1.0, -1.0 if m & 2 else 1.0, 1.0, 1.0], device="cuda")
                acc += out * sign
            out = acc * 0.25
        yv = out.cpu().numpy().astype(np.float64)
        lab = ht.cpu().numpy().astype(np.float64)
        fdn = hfd.cpu().numpy().astype(np.float64)[:, :3]
        L = np.linalg.norm(yv[:, :3], axis=1)
        nml = yv[:, :3] / np.maximum(L, 1e-30)[:, None]
        use = (L >= 0.5) & (L <= 2.0) & (np.sum(nml * fdn, axis=1) >= np.cos(np.radians(30.0)))
        e_fd = _angles(fdn, lab[:, :3])
        e_ml = _angles(np.where(use[:, None], nml, fdn), lab[:, :3])
        logged = {"workload": log_name, "steps": log_steps, "train": n_logged, "held_out": int(len(hf)),
                  "mirror_average": bool(MLP_MIRROR),
                  "label": "height function (3x3 columns of 7 cells)",
                  "fd_deg": round(float(e_fd.mean()), 4), "learned_deg": round(float(e_ml.mean()), 4),
                  "taken": round(float(use.mean()), 4),
                  "kappa_mae": round(float(np.abs(np.where(use, yv[:, 3], 0.0) - lab[:, 3]).mean()), 6),
                  "kappa_label_mean_abs": round(float(np.abs(lab[:, 3]).mean()), 6)}
    # FLOPs of one sample and step of the 27-64-64-4 network: forward 2 x 6080
    # multiply-adds; backward the weight gradients of every layer and the
    # activation gradients of the two upper ones
    macs = 27 * 64 + 64 * 64 + 64 * 4
    flops = 2 * (3 * macs - 27 * 64)
    tflops = flops * 4096 * steps / max(t2 - t1, 1e-9) / 1e12
    peak, kind = _bf16_peak()
    return theta.cpu().numpy(), {"stencils": n_stencils, "logged_stencils": logged, "steps": steps,
                                 "batch": 4096, "lr": [2e-3, 1e-5],
                                 "loss_first": float(c[0]), "loss_last100": float(c[-100:].mean()),
                                 "data_s": round(t1 - t0, 2), "train_s": round(t2 - t1, 2),
                                 "roofline": {"bound": "latency", "flops_per_sample": flops,
                                              "achieved_tflops": round(tflops, 2), "peak_tflops": peak,
                                              "peak_kind": kind, "frac": round(tflops / peak, 5),
                                              "us_per_step": round(1e6 * (t2 - t1) / max(steps, 1), 1),
                                              "limiter": "each Adam step is two dependent launches over 32 "
                                                         "blocks of 128 samples (a 4096 batch fills a fifth "
                                                         "of the SMs); the tensor cores wait on the chain"}}


def timed_run(args, w, storage_name, theta, stream, local, barrier, world, horizon=0):
    """Warm-up, then exactly args.steps timed steps of one form of the method;
    then, untimed, on to `horizon` steps in all, where the state is recorded
    for the comparison between the forms."""
    import torch

    from paper_2301_10674_gb300 import fslbm as F

    sim = F.Simulation.from_workload(w, storage=STORAGE[storage_name], stream=stream,
                                     link_mode=LINK_MODE)
    if theta is not None:
        sim.set_normal_model(theta, mirror=MLP_MIRROR)
    m0 = sim.reduce()
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
    red = sim.reduce()
    # bed topography of Section 3.2 on the final state, and its cost per call
    # through the C ABI (two kernels, a copy to the host, a synchronisation)
    bed_h = sim.bed_height()
    t0 = time.perf_counter()
    for _ in range(5):
        sim.bed_height()
    bed_ms = (time.perf_counter() - t0) / 5 * 1e3
    t0 = time.perf_counter()
    for _ in range(5):
        sim.reduce()
    red_ms = (time.perf_counter() - t0) / 5 * 1e3
    # the comparison horizon (untimed): the bed height h_b(x) is logged every
    # 10 steps on the way for its spectrum (Section 4.1)
    done = args.warmup + args.steps
    series = [sim.bed_height()]
    while done < horizon:
        k = min(10, horizon - done)
        sim.step(k)
        done += k
        series.append(sim.bed_height())
    hred = sim.reduce()
    series = np.array(series)
    spectrum = None
    if len(series) >= 2:
        dh = torch.from_numpy(series).cuda()
        psd = torch.empty_like(dh)
        rc, peak = F.fslbm_bed_spectrum(dh, len(series), w.nx, 1.0, 10.0, psd, stream.cuda_stream)
        if rc == 0:
            spectrum = {"samples": len(series), "every_steps": 10, "wavelength": float(peak[0]),
                        "period_steps": float(peak[1]), "celerity": float(peak[2]), "amplitude": float(peak[3])}
    transport = sim.transport_numbers(w.diameter)
    t = sim.get(F.FIELD_TYPE)
    phi = sim.get(F.FIELD_PHI)
    column = np.where(t == 1, 1.0, np.where(t == 2, phi, 0.0)).sum(axis=0)     # liquid volume per (y, x)
    out = {"ms": ms, "sweep_ms": sweep_ms, "sweeps": sweeps, "launches": launches, "counts": counts,
           "counts_after": counts_after, "clocks": clk, "violations": sim.violations, "m0": m0, "m1": red,
           "mh": hred, "horizon": done, "hb_end": series[-1], "spectrum": spectrum, "transport": transport,
           "column": column, "normal_stats": sim.normal_stats() if theta is not None else None,
           "bed": {"level": 0.3, "mean": round(float(bed_h.mean()), 4), "min": round(float(bed_h.min()), 4),
                   "max": round(float(bed_h.max()), 4), "ms_per_call": round(bed_ms, 3)},
           "reduce_ms_per_call": round(red_ms, 3)}
    sim.close()
    del sim
    out["ms"] = _max_over_ranks(ms, "cuda")
    return out


def _roofline(run, storage_name, ncell):
    elem = ELEM[storage_name]
    counts, counts_after = run["counts"], run["counts_after"]
    fluid = int(counts[1] + counts[2] + counts_after[1] + counts_after[2]) / 2.0
    other = ncell - fluid
    bytes_per_sweep = fluid * (54 * elem + 1) + other * 1
    sweep_s = run["sweep_ms"] / 1e3 / max(1, run["sweeps"])
    achieved = bytes_per_sweep / sweep_s / 1e9
    peak, peak_kind = _peaks()
    traffic, traffic_note = _sweep_traffic(storage_name, fluid)
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "traffic_note": traffic_note,
            "kernel": "stream-collide sweep (particle links + liquid cell pairs + interface list)",
            "bytes_per_cell": {"fluid": 54 * elem + 1, "gas_or_solid": 1},
            "bytes_per_launch": int(bytes_per_sweep), "launch_ms": round(sweep_s * 1e3, 4),
            "peak_kind": peak_kind}


def run_ours(args, world, rank, local):
    import torch

    from paper_2301_10674_gb300 import build as B

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    w = _workload(args.workload, rank)
    stream = torch.cuda.Stream()
    ncell = w.ncells

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    theta, train = None, None
    if args.normals == "mlp":
        with torch.cuda.stream(stream):
            theta, train = train_normal_model(stream, args.mlp_stencils, args.mlp_steps,
                                               log_steps=args.mlp_log_steps)
    horizon = args.error_horizon if args.compare else 0
    head = timed_run(args, w, args.storage, theta, stream, local, barrier, world, horizon)
    # the other forms, timed the same way from the same initial state: plain
    # FP32 with the finite-difference normal (the reference form), and each
    # change on its own (16-bit storage, the learned normal)
    others = {}
    if args.compare:
        for st_name, nm in COMPARE_FORMS:
            if (st_name, nm) == (args.storage, args.normals) or (nm == "mlp" and theta is None):
                continue
            others[(st_name, nm)] = timed_run(args, w, st_name, theta if nm == "mlp" else None, stream, local,
                                              barrier, world, horizon)
    base = others.get(("fp32", "fd"))
    runs = dict(others)
    runs[(args.storage, args.normals)] = head

    value = _throughput(world, ncell, args.steps, head["ms"] / 1e3)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, w, STORAGE[args.storage], theta, stream, world)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_oracle(w, steps=args.cpu_steps, warmup=1, crop_nx=args.cpu_crop, theta=theta)
        cpu = {"value": cpu["value"], "unit": UNIT, "cores": cpu["cores"], "kind": "oracle", "sample": cpu["sample"]}
    if rank != 0:
        return None

    def hdrift(r):
        return abs(r["mh"][0] - r["m0"][0]) / r["m0"][0]

    form = f"{args.storage}+{'learned' if theta is not None else 'fd'}-normal"
    comparison = None
    if base is not None:
        vb = _throughput(world, ncell, args.steps, base["ms"] / 1e3)

        def error_vs_base(r, ref=None):
            ref = base if ref is None else ref
            dcol = np.abs(r["column"] - ref["column"])
            return {"mass_drift": hdrift(r),
                    "bed_height_rms_cells": float(np.sqrt(np.mean((r["hb_end"] - ref["hb_end"]) ** 2))),
                    "bulk_ux_rel": float(abs(r["mh"][4] - ref["mh"][4]) / max(abs(ref["mh"][4]), 1e-30)),
                    "bulk_ux": float(r["mh"][4]),
                    "surface_profile_cells": {"max_abs": float(dcol.max()), "mean_abs": float(dcol.mean())},
                    "interface_cells": int(r["mh"][5])}

        def error_vs_same_normal(key, r):
            # the storage's own error: against FP32 storage with the same normal
            ref = runs.get(("fp32", key[1]))
            return None if ref is None or ref is r else error_vs_base(r, ref)

        forms = []
        for key, r in [((args.storage, args.normals), head)] + list(others.items()):
            v = _throughput(world, ncell, args.steps, r["ms"] / 1e3)
            forms.append({"form": f"{key[0]}+{'learned' if key[1] == 'mlp' else 'fd'}-normal", "value": round(v, 2),
                          "ms_per_step": round(r["ms"] / args.steps, 4), "speedup_vs_fp32_fd": round(v / vb, 4),
                          "sweep_roofline_frac": _roofline(r, key[0], ncell)["frac"],
                          "bed_spectrum": r["spectrum"],
                          "transport": {k: round(v, 8) for k, v in r["transport"].items()},
                          "error_vs_fp32_fd": None if r is base else error_vs_base(r),
                          "error_vs_fp32_same_normal": error_vs_same_normal(key, r) if key[1] == "mlp" else None})
        herr = error_vs_base(head)
        hsame = error_vs_same_normal((args.storage, args.normals), head)
        comparison = {
            "form": "fp32+fd-normal", "value": round(vb, 2), "unit": UNIT,
            "ms_per_step": round(base["ms"] / args.steps, 4), "speedup": round(value / vb, 4),
            "roofline": _roofline(base, "fp32", ncell), "clocks": base["clocks"],
            "error": {
                "horizon_steps": head["horizon"],
                "mass_drift": {"head": herr["mass_drift"], "fp32": hdrift(base)},
                "surface_profile_cells": herr["surface_profile_cells"],
                "bulk_ux_rel": herr["bulk_ux_rel"],
                "bulk_ux": {"head": float(head["mh"][4]), "fp32": float(base["mh"][4])},
                "interface_cells": {"head": herr["interface_cells"], "fp32": int(base["mh"][5])},
                # the storage alone: the head form against FP32 storage with the same normal
                "vs_fp32_same_normal": hsame,
            },
            "forms": forms,
        }
    cb = head["counts_after"]
    out = {
        "metric": _metric_name(), "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(head["ms"] / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "form": form, "lattice": [w.nx, w.ny, w.nz], "cells": ncell,
                   "spheres": w.nspheres, "spheres_nominal": w.spheres_nominal, "storage": args.storage,
                   "normals": args.normals,
                   "normal_mirror_average": bool(MLP_MIRROR) if args.normals == "mlp" else None,
                   "particle_links": {0: "library default", 1: "solid-side pass", 2: "fluid side (bed kernel)"}[LINK_MODE],
                   "cells_by_type": {"gas": int(cb[0]), "liquid": int(cb[1]), "interface": int(cb[2]),
                                     "solid": int(cb[3])},
                   "l2": f"no flush: the PDF lattice ({27 * 2 * ELEM[args.storage] * ncell / 1e9:.1f} GB incl. "
                         f"side buffer) is far larger than L2", "parallelism": f"replicas x{world}"},
        "roofline": _roofline(head, args.storage, ncell),
        "clocks": head["clocks"],
        "gpu_launches": int(head["launches"]),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "oracle_table": ORACLE_TABLE,
        "comparison": comparison,
        "learned_normal": None if theta is None else {
            "training": train,
            "evaluated": int(head["normal_stats"][0]), "taken": int(head["normal_stats"][1])},
        "checks": {"invariant_violations": int(head["violations"]), "liquid_mass": float(head["m1"][0]),
                   "interface_cells": int(head["m1"][5]), "reduce_ms_per_call": head["reduce_ms_per_call"]},
        "bed_height": head["bed"],
        "transport": {k: round(v, 8) for k, v in head["transport"].items()},
        "bed_spectrum": head["spectrum"],
    }
    return out


def run_e2e(args, w, storage, theta, stream, world):
    import torch

    from paper_2301_10674_gb300 import fslbm as F

    xyz = torch.from_numpy(np.ascontiguousarray(w.xyz)).pin_memory().numpy()
    rad = torch.from_numpy(np.ascontiguousarray(w.radius)).pin_memory().numpy()
    fix = torch.from_numpy(np.ascontiguousarray(w.fixed)).pin_memory().numpy()
    diag = torch.empty(8, dtype=torch.float64).pin_memory().numpy()
    params = F.params_from_workload(w, storage, LINK_MODE)
    bits = None if theta is None else torch.from_numpy(F.bf16_bits(theta)).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = F.fslbm_create(params, stream.cuda_stream)
    t1 = time.perf_counter()
    F._check(F.fslbm_add_spheres(h, xyz, rad, fix), "fslbm_add_spheres")
    if bits is not None:
        F._check(F.fslbm_set_normal_mirror(h, MLP_MIRROR), "fslbm_set_normal_mirror")
        F._check(F.fslbm_set_normal_model(h, bits), "fslbm_set_normal_model")
    t2 = time.perf_counter()
    t_step = t_red = 0.0
    for _ in range(args.steps):
        ta = time.perf_counter()
        F._check(F.fslbm_step(h, 1), "fslbm_step")
        tb = time.perf_counter()
        rc, out = F.fslbm_reduce(h)
        F._check(rc, "fslbm_reduce")
        diag[:] = out
        t_step += tb - ta
        t_red += time.perf_counter() - tb
    t3 = time.perf_counter()
    F.fslbm_destroy(h)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    dt = _max_over_ranks(t4 - t0, "cuda")
    phases = {"create_s": round(t1 - t0, 4), "spheres_and_weights_s": round(t2 - t1, 4),
              "steps_s": round(t3 - t2, 4), "destroy_s": round(t4 - t3, 4),
              "step_calls_s": round(t_step, 4), "reduce_calls_s": round(t_red, 4)}
    h2d = xyz.nbytes + rad.nbytes + fix.nbytes + __import__("ctypes").sizeof(params) + \
        (0 if bits is None else bits.nbytes)
    return {"value": round(_throughput(world, w.ncells, args.steps, dt), 2), "unit": UNIT,
            "h2d_bytes_per_step": round(h2d / args.steps, 1), "d2h_bytes_per_step": 64,
            "seconds": round(dt, 3), "phases": phases,
            "note": "create + particle bed (and learned-normal weights) from pinned host memory + per step "
                    "(fslbm_step, fslbm_reduce read back to host) + destroy"}


def _state(types, phi, red, u):
    """Liquid volume per (y, x) column, bulk velocity, mass, interface count and
    the velocity of the liquid cells of one state."""
    column = np.where(types == 1, 1.0, np.where(types == 2, phi, 0.0)).sum(axis=0)
    return {"column": column, "bulk_ux": float(red[4]), "mass": float(red[0]), "nifc": int(red[5]),
            "types": types, "u": u}


def run_precision_study(args):
    """Every storage / normal form of the method against the FP64 oracle on
    the 128x64x128 x-crop of the 1024x64x128 flume (the precision workload),
    after args.study_steps steps from the same initial state: mass drift,
    bulk velocity, liquid volume per column, cell types and the liquid
    velocity field. The learned-normal forms are compared with the oracle
    running the same BF16 network. Prints one JSON line."""
    import torch

    import oracle as O
    from paper_2301_10674_gb300 import build as B
    from paper_2301_10674_gb300 import fslbm as F
    from paper_2301_10674_gb300 import workloads as W

    B.build()
    torch.cuda.set_device(0)
    w = W.precision().generate().crop_x(args.study_crop)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        theta, train = train_normal_model(stream, args.mlp_stencils, args.mlp_steps,
                                               log_steps=args.mlp_log_steps)
    steps = args.study_steps
    gpu = {}
    for st_name, nm in COMPARE_FORMS:
        sim = F.Simulation.from_workload(w, storage=STORAGE[st_name], stream=stream,
                                         link_mode=LINK_MODE)
        if nm == "mlp":
            sim.set_normal_model(theta, mirror=MLP_MIRROR)
        m0 = sim.reduce()[0]
        sim.step(steps)
        st = _state(sim.get(F.FIELD_TYPE), sim.get(F.FIELD_PHI), sim.reduce(), sim.get(F.FIELD_U)[0])
        st["drift"] = abs(st["mass"] - m0) / m0
        gpu[(st_name, nm)] = st
        sim.close()
    orc = {}
    for nm in ("fd", "mlp"):
        o = O.Oracle(O.OracleParams(
            nx=w.nx, ny=w.ny, nz=w.nz, periodic=tuple(w.periodic), omega=w.omega, g=tuple(w.g), rho_gas=w.rho_gas,
            liquid_height=w.liquid_height, eps_conv=w.eps_conv, eps_normal=w.eps_normal,
            reconstruct_normal=w.reconstruct_normal, rho_p=w.rho_p, restitution=w.restitution, friction=w.friction,
            poisson=w.poisson, collision_time=w.collision_time, dem_substeps=w.dem_substeps))
        o.add_spheres(w.xyz, w.radius, w.fixed)
        if nm == "mlp":
            bits = F.bf16_bits(theta).astype(np.uint32) << 16
            o.set_mlp(bits.view(np.float32).astype(np.float64), bf16=True, mirror=MLP_MIRROR)
        m0 = o.reduce()[0]
        t0 = time.perf_counter()
        o.step(steps)
        dt = time.perf_counter() - t0
        st = _state(o.get(O.F_TYPE), o.get(O.F_PHI), o.reduce(), o.get(O.F_U)[0])
        st["drift"] = abs(st["mass"] - m0) / m0
        st["seconds"] = dt
        orc[nm] = st
        o.close()
    forms = []
    for (st_name, nm), g in gpu.items():
        r = orc[nm]
        both = (g["types"] == 1) & (r["types"] == 1)
        du = g["u"][both] - r["u"][both]
        dcol = np.abs(g["column"] - r["column"])
        forms.append({
            "form": f"{st_name}+{'learned' if nm == 'mlp' else 'fd'}-normal",
            "mass_drift": g["drift"], "oracle_mass_drift": r["drift"],
            "bulk_ux": g["bulk_ux"], "oracle_bulk_ux": r["bulk_ux"],
            "bulk_ux_rel": abs(g["bulk_ux"] - r["bulk_ux"]) / max(abs(r["bulk_ux"]), 1e-30),
            "u_liquid_rel_l2": float(np.sqrt((du ** 2).sum() / max((r["u"][both] ** 2).sum(), 1e-300))),
            "column_cells": {"max_abs": float(dcol.max()), "mean_abs": float(dcol.mean())},
            "cell_types_differing": int((g["types"] != r["types"]).sum()),
            "interface_cells": {"gpu": g["nifc"], "oracle": r["nifc"]},
        })
    return {"study": "precision forms against the FP64 oracle", "workload": w.name,
            "lattice": [w.nx, w.ny, w.nz], "spheres": w.nspheres, "steps": steps,
            "oracle_cores": O.threads(), "oracle_seconds": {k: round(v["seconds"], 1) for k, v in orc.items()},
            "learned_normal_training": train, "forms": forms}


# The oracle timed on the host cores of the GB300 machine (16 Grace cores) by
# `python bench.py --oracle-table`: the tiny flume in full, the mid flume
# and a 128-wide x-crop of the precision flume for 200 steps each. The line
# quotes it beside the live cpu_baseline.
ORACLE_TABLE = {
    "cores": 16, "host": "GB300 box (Grace)", "normal": "finite-difference",
    "rows": [
        {"workload": "tiny-64x16x32", "sample": "full lattice, 34 spheres, 1000 steps", "mlups": 4.051},
        {"workload": "mid-512x40x96", "sample": "full lattice, 1160 spheres, 200 steps", "mlups": 3.571},
        {"workload": "precision-1024x64x128", "sample": "128x64x128 x-crop, 651 spheres, 200 steps",
         "mlups": 3.858},
    ],
}


def run_oracle_table() -> dict:
    """Oracle MLUPS of the smaller workloads, each with its particle bed and
    the finite-difference normal."""
    from paper_2301_10674_gb300 import workloads as W
    rows = []
    for name, crop, steps in (("tiny", None, 1000), ("mid", None, 200), ("precision", 128, 200)):
        w = W.WORKLOADS[name]().generate()
        r = run_oracle(w, steps=steps, warmup=1, crop_nx=crop or w.nx)
        rows.append({"workload": w.name, "sample": r["sample"], "mlups": round(r["value"], 3), "cores": r["cores"],
                     "mlups_per_core": round(r["value"] / r["cores"], 4), "seconds": round(r["seconds"], 1)})
    return {"oracle_table": rows}


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
    ap.add_argument("--storage", choices=tuple(STORAGE), default="fp16")
    ap.add_argument("--normals", choices=("fd", "mlp"), default="mlp")
    ap.add_argument("--compare", action=argparse.BooleanOptionalAction, default=True,
                    help="also time plain FP32 with the finite-difference normal and the other forms")
    ap.add_argument("--error-horizon", type=int, default=300,
                    help="steps after which the forms' states are compared (untimed beyond the timed steps)")
    ap.add_argument("--mlp-stencils", type=int, default=1 << 22)
    ap.add_argument("--mlp-steps", type=int, default=40000)
    ap.add_argument("--mlp-log-steps", type=int, default=300,
                    help="steps of the mid-flume run whose logged stencils join the training (0: none)")
    ap.add_argument("--links", type=int, choices=(0, 1, 2), default=0,
                    help="particle links: 0 the library's choice, 1 pass over the solid cells, 2 fluid side")
    ap.add_argument("--mlp-mirror", action=argparse.BooleanOptionalAction, default=True,
                    help="average the learned normal over the mirror images in x and y")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=5)
    ap.add_argument("--cpu-crop", type=int, default=64)
    ap.add_argument("--ref-crop", type=int, default=64)
    ap.add_argument("--oracle-table", action="store_true",
                    help="instead of the benchmark: time the oracle on the tiny flume, the mid flume and a "
                         "128-wide crop of the precision flume (host cores)")
    ap.add_argument("--precision-study", action="store_true",
                    help="instead of the benchmark: every form against the FP64 oracle on a crop of the "
                         "1024x64x128 flume")
    ap.add_argument("--study-steps", type=int, default=500)
    ap.add_argument("--study-crop", type=int, default=128)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    global LINK_MODE, MLP_MIRROR
    LINK_MODE = args.links
    MLP_MIRROR = args.mlp_mirror
    world, rank, local = _dist()
    if args.precision_study:
        print(json.dumps(run_precision_study(args)), flush=True)
        return
    if args.oracle_table:
        print(json.dumps(run_oracle_table()), flush=True)
        return
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
