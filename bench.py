#!/usr/bin/env python
"""Throughput benchmark of the two-range pseudopotential lattice Boltzmann
step (Fei et al., arXiv:1806.06943) on GB300.

Workload (default, ``laplace_sweep_24``): the batched Laplace sweep, 24
periodic lattices of sides 128..384 (droplet radii 10..45 at viscosity ratios
1, 3 and 10, tau_c = 1), 1,520,640 sites, FP32 offset populations, all
lattices advanced by one launch per kernel.  One benchmark step = one time
step of the whole batch (density pass + fused force/collide/stream kernel).
The L2 cache is flushed (256 MiB overwrite) before every timed step, outside
the timed intervals; steps are timed on the device with CUDA events.

Metric: two-species MLUPS = lattice sites x time steps / s / 1e6, where one
site update advances both species.  With --gpus N (torchrun), every rank
advances its own copy of the batch (weak scaling, no data-path collective);
the value is the sum over ranks divided by the slowest rank's time.

Roofline: the step kernel's algorithmic bytes (the populations read and
written once: 144 B per node in FP32, 288 B in FP64) per launch over its
CUDA-event time, against the measured copy bandwidth; the design's own
byte count (160 B per node in FP32, with the reference densities) beside
it.  The FP64 kernel is bound by the FP64 pipe and is reported against the
device's measured FP64 FMA rate.

Side legs (skipped with --quick): the Laplace fit of the sweep after 20000
steps, the same batch in FP64, the 4096x4096 dense emulsion in FP32 and
FP64, an end-to-end job through the public API with host buffers, the
adjoint, and the CPU oracle timed on a bounded sample on one and on every
host core.
``--impl reference`` times the CPU oracle alone as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

C6 = dict(G_AB=3.0, G1=-7.4, G2=6.4)
FLUSH_BYTES = 256 << 20
# Algorithmic bytes per node update (FP32 offset / FP64 plain): the 2 x 9
# populations read once and written once.  The roofline fraction is taken
# on these.
FLOOR_BYTES = {1: 144, 0: 288}
# Bytes each kernel of this design moves per node and launch, reported beside
# the floor: the FP32 form also reads the node's 2 reference densities and
# writes its 2 densities (the next step's references).
BYTES_FUSED = {1: 160, 0: 288}     # one-pass: 18 pops read + 18 written (+ 2 reference rho read, 2 written)
BYTES_COLLIDE = {1: 160, 0: 304}   # two-pass fused kernel: 18 pops read + 18 written + 2 rho read (+ 2 reference rho read)
BYTES_DENSITY = {1: 88, 0: 160}    # density pass: 18 pops read + 2 rho written (+ 2 reference rho read)
# FP64 operations per node of the FP64 one-pass kernel (k_fused<double, 8>):
# DADD + DMUL + 2 DFMA thread instructions per node (344 + 236 + 2 x 61.25),
# counted by ncu on the 512^2 dense emulsion
# (profiles/k_fused_fp64_dense_emulsion_512.md); FP64 pipe instructions per
# node (DADD + DMUL + DFMA) beside it.
FP64_FLOPS_PER_NODE = 702.6
FP64_PIPE_OPS_PER_NODE = 641.3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--quick", action="store_true", help="main leg only")
    ap.add_argument("--workload", default="laplace_sweep_24",
                    choices=["laplace_sweep_24", "dense_emulsion_4096", "dense_emulsion_2048", "dense_emulsion_512"],
                    help="main-leg workload (the dense emulsions are single periodic lattices)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--mode", default="tma", choices=["tma", "fused", "launch"],
                    help="time step as one pass (fused) or density pass + fused kernel (launch)")
    ap.add_argument("--tile-height", type=int, default=8, choices=[2, 4, 8])
    return ap.parse_args()


# ---- distributed helpers (host logic, also used by the CPU tests) -----------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, local, world


def init_dist(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---- workloads ----------------------------------------------------------------

def sweep_fields():
    from paper_1806_06943_gb300 import workloads as W
    specs = W.laplace_sweep_specs()
    fields = [W.droplet(s["nx"], s["ny"], s["R"], seed=W.BASE_SEED + 1 + i) for i, s in enumerate(specs)]
    return specs, fields


def dense_emulsion(n):
    """n x n periodic emulsion, radii U[8, 20], target area fraction 0.6,
    dispersed/continuous viscosity ratio 5 (tau_d = 3, tau_c = 1)."""
    from paper_1806_06943_gb300 import workloads as W
    rho, _, radii, phi = W.random_emulsion(n, n, 0.6, 8.0, 20.0, seed=W.BASE_SEED + 4)
    return [dict(nx=n, ny=n, tau=(3.0, 1.0), R=0.0)], [rho], {"phi_achieved": phi, "droplets": len(radii)}


def make_batch(lb, specs, fields, precision, stream):
    b = lb.Batch([dict(nx=s["nx"], ny=s["ny"], tau=s["tau"]) for s in specs], precision=precision,
                 stream=stream, **C6)
    for i, (s, r) in enumerate(zip(specs, fields)):
        b.set_fields(i, r)
        if s.get("R", 0.0) > 0.0:
            b.set_probe(i, s["nx"] / 2, s["ny"] / 2, s["R"])
    return b


# ---- clocks ----------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = ("lb_kernels.cuh", "lb_vops.cuh", "lb_tma.cu")


def kernel_source_sha1() -> str:
    """SHA-1 over the kernel sources (lb_kernels.cuh, lb_vops.cuh, then lb_tma.cu)."""
    import hashlib
    h = hashlib.sha1()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1806_06943_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_traffic(workload: str, kernel: str):
    """DRAM bytes per launch of a step kernel from the committed ncu summary
    (profiles/traffic.json: a list of entries), if one was taken on this
    workload, on this kernel and on the current kernel sources; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            entries = json.load(f)
        sha = kernel_source_sha1()
        for d in entries:
            if d.get("workload") == workload and d.get("kernel") == kernel and d.get("kernel_source_sha1") == sha:
                return float(d["bytes_per_launch"])
    except Exception:
        pass
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def hbm_roofline(kname, units, ms, peak, peak_kind, floor_b, design_b, traffic):
    """Roofline of an HBM-bound step kernel: achieved = algorithmic bytes per
    node (the populations read and written once) x nodes per launch / the
    launch's CUDA-event time; the design's own byte count beside it."""
    ach = floor_b * units / (ms * 1e-3) / 1e9
    des = design_b * units / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kname, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs (burst)",
            "algorithmic_bytes_per_site": floor_b, "units_per_launch": units, "ms_per_launch": ms,
            "design_bytes_per_site": design_b, "design_achieved": des, "design_frac": des / peak}


def alu_roofline(kname, units, ms, peak_tflops, hbm_peak):
    """Roofline of the FP64 step kernel, bound by the FP64 pipe: FP64
    operations per node (ncu count) x nodes / launch time against the
    measured FP64 FMA rate of the device."""
    ach = FP64_FLOPS_PER_NODE * units / (ms * 1e-3) / 1e12 if FP64_FLOPS_PER_NODE else None
    return {"bound": "alu", "kernel": kname, "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": (ach / peak_tflops) if (ach and peak_tflops) else None, "traffic": None,
            "peak_source": "measured FP64 FMA throughput of this device (lb_device_fp64_peak)",
            "flops_per_site": FP64_FLOPS_PER_NODE, "units_per_launch": units, "ms_per_launch": ms,
            "fp64_pipe_frac": FP64_PIPE_OPS_PER_NODE * units / (ms * 1e-3) / (peak_tflops * 1e12 / 2),
            "hbm_frac_floor": FLOOR_BYTES[0] * units / (ms * 1e-3) / 1e9 / hbm_peak}


# ---- CPU oracle timing -------------------------------------------------------------

def oracle_sample(target_s: float, threads: int = 1):
    """The oracle advancing lattice 0 of the sweep (128x128, R=10, ratio 1)
    on `threads` host threads (its OpenMP row loops) for as many steps as fit
    in about target_s seconds; returns (MLUPS, description, steps, threads)."""
    import oracle
    from paper_1806_06943_gb300 import workloads as W
    used = oracle.set_threads(threads)
    s0 = W.laplace_sweep_specs()[0]
    rho = W.droplet(s0["nx"], s0["ny"], s0["R"], seed=W.BASE_SEED + 1)
    sim = oracle.OracleSim(s0["nx"], s0["ny"], tau=s0["tau"], **C6)
    sim.set_fields(rho)
    t0 = time.perf_counter()
    sim.step(20)
    dt = time.perf_counter() - t0
    n = max(20, int(target_s / max(dt, 1e-6) * 20))
    t0 = time.perf_counter()
    sim.step(n)
    dt = time.perf_counter() - t0
    sites = s0["nx"] * s0["ny"]
    return (sites * n / dt / 1e6,
            f"lattice 0 of the sweep ({s0['nx']}x{s0['ny']}, R={s0['R']:g}), {n} steps, {dt:.1f} s, {used} threads",
            n, used)


def run_reference(args):
    rank, local, world = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1806_06943_gb300 import workloads as W
    cores = oracle.set_threads(os.cpu_count() or 1)   # every host core (OpenMP row loops)
    s0 = W.laplace_sweep_specs()[0]
    rho = W.droplet(s0["nx"], s0["ny"], s0["R"], seed=W.BASE_SEED + 1)
    sim = oracle.OracleSim(s0["nx"], s0["ny"], tau=s0["tau"], **C6)
    sim.set_fields(rho)
    steps_per = 20 * cores   # each benchmark step: 20 time steps per core of lattice 0 (bounded sample)
    for _ in range(args.warmup):
        sim.step(steps_per)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.step(steps_per)
    dt = time.perf_counter() - t0
    sites = s0["nx"] * s0["ny"]
    v = sites * steps_per * args.steps / dt / 1e6
    out = {
        "impl": "reference", "metric": "2-species MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "laplace_sweep_24",
                   "sample": f"lattice 0 (128x128, R=10, ratio 1), {steps_per} time steps per step",
                   "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"lattice 0 of the sweep, {steps_per} time steps per benchmark step, "
                                   f"{cores} threads"},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# ---- GPU arm ------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        args.warmup = 3
    rank, local, world = dist_env()
    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = torch.device("cuda", local)
    from paper_1806_06943_gb300 import build
    if rank == 0:
        build.build()
    barrier(dist)
    from paper_1806_06943_gb300 import lb

    stream = torch.cuda.Stream(device=dev)
    sptr = stream.cuda_stream
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    peak, peak_kind = measured_peaks()
    fp64_peak = lb.device_fp64_peak(4096)

    extra_cfg = {}
    if args.workload == "laplace_sweep_24":
        specs, fields = sweep_fields()
    else:
        specs, fields, extra_cfg = dense_emulsion(int(args.workload.rsplit("_", 1)[1]))
    sites = sum(s["nx"] * s["ny"] for s in specs)
    prec = lb.LB_FP32 if args.precision == "fp32" else lb.LB_FP64
    b = make_batch(lb, specs, fields, prec, sptr)
    if args.mode == "tma" and prec == lb.LB_FP64:
        args.mode = "fused"          # the TMA-staged step is FP32 only
    mode = {"tma": lb.LB_MODE_TMA, "fused": lb.LB_MODE_FUSED, "launch": lb.LB_MODE_LAUNCH}[args.mode]
    b.set_config(mode, args.tile_height)
    one_pass = mode in (lb.LB_MODE_FUSED, lb.LB_MODE_TMA)
    kbytes = BYTES_FUSED if one_pass else BYTES_COLLIDE
    kname = (f"k_fused_tma<{args.tile_height}>" if mode == lb.LB_MODE_TMA else
             ("k_fused" if mode == lb.LB_MODE_FUSED else "k_collide")
             + f"<{'float' if prec else 'double'}, {args.tile_height}>")

    # warm-up (untimed), then the timed region: K steps, barrier + sync on both sides
    b.profile(args.warmup, flush.data_ptr(), FLUSH_BYTES)
    clocks = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    torch.cuda.synchronize()
    barrier(dist)
    clocks.start()
    t_wall0 = time.perf_counter()
    ms = b.profile(args.steps, flush.data_ptr(), FLUSH_BYTES)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier(dist)
    # keep sampling clocks over a sustained stretch of the same kernels
    b.step(2048)
    b.synchronize()
    clk = clocks.stop()
    obs = b.observables()

    ms_step = max_over_ranks(dist, ms[2], dev)
    value = sum_over_ranks(dist, sites, dev) / (ms_step * 1e-3) / 1e6
    gpu_launches = (1 if one_pass else 2) * args.steps

    out = {
        "metric": "2-species MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == lb.LB_FP32 else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "lattices": len(specs), "sites": sites,
                   "sizes": ("128^2..384^2, R 10..45, mu_d/mu_c 1, 3, 10 (tau_c = 1)"
                             if args.workload == "laplace_sweep_24" else
                             "periodic emulsion, R U[8,20], phi 0.6, mu_d/mu_c 5"), **extra_cfg,
                   "precision": ("fp32 offset populations (per-node reference density), fp64 reductions"
                                 if prec == lb.LB_FP32 else "fp64 populations"),
                   "couplings": C6, "l2": "flushed (256 MiB write) before every timed step",
                   "timing": "CUDA events per kernel on the launching stream", "parallelism": f"replicas x{world}"},
        "clocks": clk,
        "gpu_launches": gpu_launches,
        "roofline": (hbm_roofline(kname, sites, ms[1], peak, peak_kind, FLOOR_BYTES[prec], kbytes[prec],
                                  kernel_traffic(args.workload, kname))
                     if prec == lb.LB_FP32 else alu_roofline(kname, sites, ms[1], fp64_peak, peak)),
        "mode": args.mode,
        "wall_s_timed": t_wall,
        "observables_after": {"finite": all(o["finite"] == 1.0 for o in obs)},
    }

    if not args.quick and args.workload == "laplace_sweep_24" and prec == lb.LB_FP32:
        # sustained rate through the public step call (CUDA graphs, no flush)
        b.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            b.step(256)
            ev1.record(stream)
        ev1.synchronize()
        out["graph_sustained_mlups"] = sites * 256 / (ev0.elapsed_time(ev1) * 1e-3) / 1e6

        # two-pass breakdown of the same batch: density pass + fused kernel
        b.set_config(lb.LB_MODE_LAUNCH, 4)
        b.profile(3, flush.data_ptr(), FLUSH_BYTES)
        m2 = b.profile(max(20, args.steps // 2), flush.data_ptr(), FLUSH_BYTES)
        out["two_pass"] = {"mlups": sites / (m2[2] * 1e-3) / 1e6,
                           "density_ms": m2[0], "density_gbs": BYTES_DENSITY[1] * sites / (m2[0] * 1e-3) / 1e9,
                           "collide_ms": m2[1], "collide_gbs": BYTES_COLLIDE[1] * sites / (m2[1] * 1e-3) / 1e9,
                           "collide_frac": BYTES_COLLIDE[1] * sites / (m2[1] * 1e-3) / 1e9 / peak}

        # autotuned execution configuration (mode, tile height) and its sustained rate
        tuned_ms = b.autotune(64, None)
        tmode, tyh = b.config()
        b.synchronize()
        ev0.record(stream)
        b.step(256)
        ev1.record(stream)
        ev1.synchronize()
        out["autotuned"] = {"mode": ["launch", "persistent", "fused", "tma"][tmode], "tile_height": tyh,
                            "trial_ms_per_step": tuned_ms,
                            "sustained_mlups": sites * 256 / (ev0.elapsed_time(ev1) * 1e-3) / 1e6}

        # the sweep's own observable: 20000 steps of all 24 drops (FP32, the
        # configured mode), then the Laplace law dp = gamma / R_eff + c fitted
        # per viscosity ratio
        bl = make_batch(lb, specs, fields, lb.LB_FP32, sptr)
        bl.set_config(mode, args.tile_height)
        t0 = time.perf_counter()
        bl.step(20000)
        obs_l = bl.observables()
        t_l = time.perf_counter() - t0
        fits = {}
        for ratio in sorted({sp["ratio"] for sp in specs}):
            pts = [(1.0 / o["R_eff"], o["dp"]) for sp, o in zip(specs, obs_l) if sp["ratio"] == ratio]
            xs, ys = [p[0] for p in pts], [p[1] for p in pts]
            n_, mx, my = len(xs), sum(xs) / len(xs), sum(ys) / len(ys)
            sxx = sum((x - mx) ** 2 for x in xs)
            gamma = sum((x - mx) * (y - my) for x, y in zip(xs, ys)) / sxx
            c0 = my - gamma * mx
            ss_res = sum((y - gamma * x - c0) ** 2 for x, y in zip(xs, ys))
            ss_tot = sum((y - my) ** 2 for y in ys)
            fits[f"ratio_{ratio:g}"] = {"gamma": gamma, "intercept": c0, "r2": 1 - ss_res / ss_tot, "drops": n_}
        out["laplace_fit_20k"] = {"steps": 20000, "seconds": t_l, "precision": "fp32", "fits": fits,
                                  "finite": all(o["finite"] == 1.0 for o in obs_l)}
        del bl

        # FP64 on the same batch
        b64 = make_batch(lb, specs, fields, lb.LB_FP64, sptr)
        b64.set_config(lb.LB_MODE_FUSED if mode == lb.LB_MODE_TMA else mode, 8)
        b64.profile(3, flush.data_ptr(), FLUSH_BYTES)
        k64 = max(10, args.steps // 4)
        ms64 = b64.profile(k64, flush.data_ptr(), FLUSH_BYTES)
        out["fp64_same_workload"] = {
            "mlups": sites / (ms64[2] * 1e-3) / 1e6, "ms_per_step": ms64[2], "steps": k64,
            "kernel_ms": ms64[1], "density_ms": ms64[0],
            "roofline": alu_roofline("k_fused<double, 8>", sites, ms64[1], fp64_peak, peak),
        }
        out["fp32_over_fp64"] = value / out["fp64_same_workload"]["mlups"]
        del b64

        # large dense emulsion, 4096^2, FP32 offset and FP64
        from paper_1806_06943_gb300 import workloads as W
        rho4k, _, radii, phi = W.random_emulsion(4096, 4096, 0.6, 8.0, 20.0, seed=W.BASE_SEED + 4)
        big = {"phi_achieved": phi, "droplets": len(radii)}
        for prec, name in ((lb.LB_FP32, "fp32"), (lb.LB_FP64, "fp64")):
            L = lb.Lattice(4096, 4096, tau=(3.0, 1.0), precision=prec, stream=sptr, **C6)
            L.set_fields(rho4k)
            n4 = 4096 * 4096
            k = 20 if prec == lb.LB_FP32 else 8
            big_mode = mode if prec == lb.LB_FP32 else lb.LB_MODE_FUSED
            L.set_config(big_mode, args.tile_height)
            L.profile(3, flush.data_ptr(), FLUSH_BYTES)
            m = L.profile(k, flush.data_ptr(), FLUSH_BYTES)
            L.set_config(lb.LB_MODE_LAUNCH, 4)
            L.profile(2, flush.data_ptr(), FLUSH_BYTES)
            m2 = L.profile(k, flush.data_ptr(), FLUSH_BYTES)
            bk = (f"k_fused_tma<{args.tile_height}>" if big_mode == lb.LB_MODE_TMA else
                  f"k_fused<{'float' if prec else 'double'}, {args.tile_height}>")
            big[name] = {"mode": ["launch", "persistent", "fused", "tma"][big_mode], "tile_height": args.tile_height,
                         "mlups": n4 / (m[2] * 1e-3) / 1e6, "ms_per_step": m[2], "steps": k,
                         "roofline": (hbm_roofline(bk, n4, m[1], peak, peak_kind, FLOOR_BYTES[prec], BYTES_FUSED[prec],
                                                   kernel_traffic("dense_emulsion_4096", bk))
                                      if prec == lb.LB_FP32 else alu_roofline(bk, n4, m[1], fp64_peak, peak)),
                         "two_pass_mlups": n4 / (m2[2] * 1e-3) / 1e6, "collide_ms": m2[1], "density_ms": m2[0],
                         "collide_frac_floor": FLOOR_BYTES[prec] * n4 / (m2[1] * 1e-3) / 1e9 / peak,
                         "collide_frac_design": BYTES_COLLIDE[prec] * n4 / (m2[1] * 1e-3) / 1e9 / peak}
            del L
        out["large_dense_4096"] = big

        # the 3-D extension: a periodic 160^3 emulsion of spheres (radius 8,
        # viscosity ratio 5), FP32 offsets and FP64, two launches per step
        three = {}
        n3 = 160
        z3, y3, x3 = [a.astype(np.float64) for a in np.meshgrid(np.arange(n3), np.arange(n3), np.arange(n3),
                                                                   indexing="ij")]
        m3 = np.zeros((n3, n3, n3), dtype=bool)
        for cz in range(10, n3, 20):
            for cy in range(10, n3, 20):
                for cx in range(10, n3, 20):
                    m3 |= (x3 - cx) ** 2 + (y3 - cy) ** 2 + (z3 - cz) ** 2 < 64.0
        rho3 = np.empty((2, n3, n3, n3))
        rho3[0] = np.where(m3, 1.0, 0.03)
        rho3[1] = np.where(m3, 0.03, 1.0)
        del x3, y3, z3
        for prec, name in ((lb.LB_FP32, "fp32"), (lb.LB_FP64, "fp64")):
            L3 = lb.Lattice3(n3, n3, n3, tau=(3.0, 1.0), precision=prec, stream=sptr, **C6)
            L3.set_fields(rho3)
            L3.profile(3, flush.data_ptr(), FLUSH_BYTES)
            m = L3.profile(10 if prec == lb.LB_FP32 else 4, flush.data_ptr(), FLUSH_BYTES)
            nodes = n3 ** 3
            floor3 = 2 * 38 * (4 if prec == lb.LB_FP32 else 8)
            three[name] = {"mlups": nodes / (m[2] * 1e-3) / 1e6, "ms_per_step": m[2], "density_ms": m[0],
                           "collide_ms": m[1], "algorithmic_bytes_per_site": floor3,
                           "step_frac_floor": floor3 * nodes / (m[2] * 1e-3) / 1e9 / peak,
                           "phi_achieved": float(m3.mean())}
            del L3
        out["three_d_160"] = three
        del rho3, m3

        # end to end through the public API with host buffers: per e2e step,
        # upload every lattice's initial fields from pinned host memory, run
        # 100 time steps, read back the observables of all 24 lattices
        pinned = [torch.from_numpy(f).pin_memory().numpy() for f in fields]
        S = 100
        e2e_iters = 3
        be = lb.Batch([dict(nx=s["nx"], ny=s["ny"], tau=s["tau"]) for s in specs], precision=lb.LB_FP32,
                      stream=sptr, **C6)
        be.set_config(mode, args.tile_height)
        for i in range(len(specs)):
            be.set_fields(i, pinned[i])
        be.step(S)
        be.observables()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_iters):
            for i in range(len(specs)):
                be.set_fields(i, pinned[i])
            be.step(S)
            be.observables()
        dt = time.perf_counter() - t0
        h2d = sum(f.nbytes for f in pinned)
        out["e2e"] = {"value": sites * S * e2e_iters / dt / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": 24 * 16 * 8,
                      "step": f"upload fields of all 24 lattices + {S} time steps + observables readback"}
        out["gpu_launches"] = gpu_launches
        del be

        # adjoint: gradient of mu_r for the 512 x 128 channel emulsion, 5000
        # steps, checkpoints every 250: FP32 forward and recomputation with the
        # FP64 adjoint (the calibration configuration), and the FP64 forward
        from paper_1806_06943_gb300 import workloads as W
        rho_c, _, _, phi_c = W.hex_emulsion(512, 128, 0.5, R=12.0, spread=2.0, gap=3.0, walls=True,
                                            seed=W.BASE_SEED + 3)
        adj = {"steps": 5000, "ckpt_every": 250, "phi_achieved": phi_c, "theta": "G_AB, G1, G2, tau_A, tau_B"}
        for prec, name in ((lb.LB_FP32, "fp32_forward"), (lb.LB_FP64, "fp64_forward")):
            Lc = lb.Lattice(512, 128, tau=(1.0, 1.0), g=(1e-6, 0.0), walls=1, wall_mode=1, wall_rho=(0.03, 1.0),
                            precision=prec, stream=sptr, **C6)
            Lc.set_config(lb.LB_MODE_TMA if prec == lb.LB_FP32 else lb.LB_MODE_FUSED, 8)
            Lc.set_fields(rho_c)
            t0 = time.perf_counter()
            Jc, dJc = Lc.grad(5000, 250, lb.LB_OBJ_MU_R)
            tg = time.perf_counter() - t0
            adj[name] = {"mu_r": Jc, "dmu_r_dtheta": [float(v) for v in dJc], "seconds": tg,
                         "forward_equivalent_mlups": 512 * 128 * 5000 / tg / 1e6}
            del Lc
        g32, g64 = adj["fp32_forward"]["dmu_r_dtheta"], adj["fp64_forward"]["dmu_r_dtheta"]
        adj["fp32_vs_fp64_max_rel"] = max(abs(x / y - 1) for x, y in zip(g32, g64))
        out["adjoint_channel_512x128"] = adj

        # CPU oracle on a bounded sample (rank 0 only)
        if rank == 0 and world == 1:
            ncores = os.cpu_count() or 1
            v1, sample1, _, _ = oracle_sample(8.0, 1)
            vn, samplen, _, used = oracle_sample(8.0, ncores)
            out["cpu_baseline"] = {"value": vn, "unit": "MLUPS", "cores": used, "kind": "oracle", "sample": samplen,
                                   "one_core": {"value": v1, "sample": sample1}, "nproc": ncores}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
