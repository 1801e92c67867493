"""Benchmark of the fused WENO5 / Lax-Friedrichs / SSP-RK3 step on GB300.

Default workload: the large forward-throughput configuration -- 8192 x 8192 periodic grid, gamma 1.4,
FP32 state with 5 fields (rho, rho u, rho v, tau, level set phi), seeded density/pressure blobs plus a
p = 100 blast, level-set burning speed 0.05. One benchmark step is one SSP-RK3 time step of the whole
grid: three fused stage launches (flux split, WENO5 in x and y, sources, level-set Hamiltonian, RK
blend, the next stage's Lax-Friedrichs speeds, the next step's CFL speed and the FP64 totals of the
new state). The state (1.34 GB per copy) is far larger than L2, so no flush is needed.

Output: one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle instead, on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK3 step"
UNIT = "cell-updates/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, world


def max_over_ranks(x: float, world: int) -> float:
    """The largest value of x over the ranks of the default process group (the slowest replica's time);
    x itself on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput of `world` replicas that each processed units_per_rank units, timed by the
    slowest one (weak scaling)."""
    return world * units_per_rank / seconds


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"hydro_bench_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as f:
            return self.summarise(f)

    @staticmethod
    def summarise(lines):
        """Median and maximum SM clock and the throttle reasons seen, from nvidia-smi CSV lines (no header,
        no units) of the FIELDS query; None without a sample."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            v = [s.strip() for s in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                mx.append(float(v[2]))
            except ValueError:
                continue
            for n, flag in zip(names, v[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


SLOWDOWN_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(clk, stuck_below: float = 0.8):
    """Why a timed region's clock record rejects its number, else None: a hardware or thermal slowdown
    active during the region, or the median SM clock well below the maximum with no reason active (a clock
    locked by an earlier user). A power cap alone (sw_power_cap) keeps the number; it stays in `reasons`."""
    if not clk:
        return None
    bad = [r for r in clk["reasons"] if r in SLOWDOWN_REASONS]
    if bad:
        return ",".join(bad)
    if not clk["reasons"] and clk["sm_mhz"] < stuck_below * clk["sm_max_mhz"]:
        return f"sm clock {clk['sm_mhz']:.0f} of {clk['sm_max_mhz']:.0f} MHz with no reason"
    return None


WORKLOADS = {
    # name: (generator, default dtype, description)
    "blobs_blast_8192": ("large forward throughput: 8192^2 periodic, 5 fields, blobs + blast", "f32"),
    "blobs_blast_4096": ("the same state generator at 4096^2 (profiling case)", "f32"),
    "rayleigh_taylor_1024x2048": ("axisymmetric Rayleigh-Taylor with gravity and level set", "f32"),
    "advected_wave_128": ("128^2 periodic advected density wave (plain method)", "f64"),
    "quadrant_ensemble_64": ("64 quadrant Riemann problems of uneven sizes, batched", "f32"),
    "fourier_256_adjoint": ("256^2 Fourier-mode state, 200 steps, checkpoints every 20, adjoint sweep", "f64"),
}


def workload(name: str):
    from paper_1507_08549_gb300 import workloads as wl
    if name == "blobs_blast_8192":
        return wl.blobs_blast(8192)
    if name == "blobs_blast_4096":
        return wl.blobs_blast(4096)
    if name == "rayleigh_taylor_1024x2048":
        return wl.rayleigh_taylor(1024, 2048)
    if name == "advected_wave_128":
        return wl.advected_wave(128)
    if name == "quadrant_ensemble_64":
        return wl.quadrant_ensemble(64)
    if name == "fourier_256_adjoint":
        return wl.fourier_modes(256)[0]
    raise SystemExit(f"unknown workload {name}")


def crop(prob, cap: int):
    """The first min(cap, ny) rows and min(cap, nx) columns of a workload's state as a problem of their
    own (same spacing, generator and physics; the crop's faces keep the workload's boundary kinds)."""
    nx, ny = min(cap, prob.nx), min(cap, prob.ny)
    return prob.with_(nx=nx, ny=ny, x1=prob.x0 + nx * prob.dx, y1=prob.y0 + ny * prob.dy,
                      U0=np.ascontiguousarray(prob.U0[:, :ny, :nx]))


def cpu_baseline(prob, seconds: float = 10.0):
    """Time the FP64 oracle, as it stands, on all host cores on a crop of at most 2048 x 2048 cells of
    the workload until about `seconds` of wall time are spent."""
    import oracle
    sub = crop(prob, 2048)
    oracle.build()
    U = sub.U0
    steps, t0 = 0, time.perf_counter()
    while True:
        U, _, _ = oracle.step(sub, U, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": sub.cells * steps / el, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"{sub.nx}x{sub.ny} crop of the workload, {steps} FP64 RK3 steps, {el:.1f} s wall"}


def run_reference(args):
    rank, world = _dist()
    if rank != 0:
        return 0
    prob = workload(args.workload)
    if isinstance(prob, list):
        prob = max(prob, key=lambda q: q.cells)
    # each reference "step" is one oracle step of the crop; warm-up steps are untimed
    import oracle
    sub = crop(prob, 1024)
    oracle.build()
    U = sub.U0
    for _ in range(args.warmup):
        U, _, _ = oracle.step(sub, U, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, _, _ = oracle.step(sub, U, 1)
    el = time.perf_counter() - t0
    value = sub.cells * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample": f"{sub.nx}x{sub.ny} crop", "cells": sub.cells},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": f"{sub.nx}x{sub.ny} crop of {args.workload}, {args.steps} FP64 RK3 steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# Measured DRAM traffic of the stage kernel (dram__bytes_read.sum + dram__bytes_write.sum from one ncu
# capture, averaged over the three stage launches of one RK3 step, per cell), per tile shape, valid only for
# the kernel source it was captured on: `stage_traffic_per_cell` returns None once stage_kernel.cuh has
# changed (its SHA-256 differs from the one recorded here) or for a tile shape without a capture.
STAGE_TRAFFIC = {
    "stage_kernel_sha256": "c08adba5d5228e143579175afc4da42cc30bce79ec17b78989c6259662d96ba8",
    # bytes per cell and launch of the 8192^2 blobs + blast state (5 fields, FP32), by tile "TXxTY"
    "bytes_per_cell_launch_f32_nf5": {
        # reads 1840.4, 3311.4, 3181.0 MB, writes 1312.5, 1327.4, 1308.2 MB
        "60x15": (1840.402176 + 3311.394560 + 3181.026048 + 1312.472064 + 1327.383040 + 1308.198912) * 1e6
        / 3.0 / (8192 * 8192),
        # reads 1357.5, 2709.2, 2706.5 MB, writes 1301.5, 1313.1, 1299.7 MB
        "60x30": (1357.523712 + 2709.227776 + 2706.496000 + 1301.529856 + 1313.074432 + 1299.652352) * 1e6
        / 3.0 / (8192 * 8192),
    },
    "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none "
               "-k regex:stage_kernel -s 9 -c 3 python bench.py --workload blobs_blast_8192 --steps 2 --warmup 3 "
               "--quick --no-cpu-baseline --variant V (1 pass per launch)",
}


def stage_kernel_sha256() -> str:
    import hashlib
    path = os.path.join(ROOT, "paper_1507_08549_gb300", "csrc", "stage_kernel.cuh")
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def stage_traffic_per_cell(tile: str = "60x15"):
    """Measured bytes per cell and stage launch of the current stage kernel source with tile shape
    "TXxTY", else None."""
    if stage_kernel_sha256() != STAGE_TRAFFIC["stage_kernel_sha256"]:
        return None
    return STAGE_TRAFFIC["bytes_per_cell_launch_f32_nf5"].get(tile)


# FP32 arithmetic operations per cell and RK stage (one per rounded operation, a fused multiply-add counted
# once). Per cell, one hydro component and one direction (the method: one point's flux and split, that
# point's two triplets -- one per reconstruction direction -- and one face): flux 3 + split 2, 2 triplets x 23
# (smoothness data, weights and candidate values of one reconstruction direction), one face x 15 (two weighted
# sums of 7 and their sum), one difference x 2, and half an accumulation (the y pass adds to the x pass's
# value): 68.5 ops, 8 such lines per cell (4 components, 2 directions). The level set per direction: one
# difference x 2, one triplet x 25 (shared by both one-sided derivatives), one cell x 14: 41 ops, 2 directions.
# Primitives of the cell: 8 ops. The cell phase (sources, RK blend, next stage's speeds, totals): 61 ops with
# the level-set Hamiltonian, 40 without.
METHOD_HYDRO_LINE_CELL = 5 + 2 * 23 + 15 + 2 + 0.5
METHOD_PHI_LINE_CELL = 2 + 25 + 14
METHOD_PRIMS_CELL = 8.0


def method_ops_per_cell_stage(F):
    """The method's own operation count per cell and stage (no tile or line halos)."""
    return 8 * METHOD_HYDRO_LINE_CELL + METHOD_PRIMS_CELL + (2 * METHOD_PHI_LINE_CELL + 61.0 if F == 5 else 40.0)


# What the kernel spends, its line halos included: a 15-cell line reads 21 points and forms 36 triplets
# (18 per reconstruction direction) and 16 faces, so a hydro line costs 21 x 5 + 36 x 23 + 16 x 15 + 15 x 2
# + 7.5 = 1210.5 ops (80.7 per cell) and a level-set line 20 x 2 + 18 x 25 + 15 x 14 = 700 (46.7 per cell);
# the primitives are formed on the halo box (12.3 per cell).
def kernel_ops_per_cell_stage(F):
    return 8 * 80.7 + 12.3 + (2 * 46.7 + 61.0 if F == 5 else 40.0)


def roofline(F, B, cells, avg_launch_ms, sm_mhz=None, alu=False, traffic=None):
    """Roofline of the stage kernel. HBM: algorithmic bytes per launch = 8 F B per cell per step (stage 1
    reads U^n and writes U^(1); stages 2 and 3 read U^n and the stage input and write) over 3 launches.
    ALU (FP32): the method's operations per launch (method_ops_per_cell_stage, no halo recomputation)
    against 152 SMs x 128 FP32 lanes x SM clock; the kernel's own count (halos included) is reported beside
    it as kernel_ops_per_cell."""
    alg_bytes_per_launch = 8 * F * B * cells / 3.0
    achieved = alg_bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "peak_kind": peak_kind, "kernel": "stage_kernel", "avg_launch_ms": avg_launch_ms,
           "alg_bytes_per_launch": alg_bytes_per_launch}
    if not alu:
        return hbm, None
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_mhz or 2070.0
    ops = method_ops_per_cell_stage(F) * cells
    a = ops / (avg_launch_ms * 1e-3) / 1e12
    pk = sms * 128 * mhz * 1e6 / 1e12
    roof = {"bound": "alu", "achieved": a, "peak": pk, "unit": "T FP32 ops/s (FMA = 1)", "frac": a / pk,
            "traffic": traffic, "peak_kind": f"derived: {sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz (sampled)",
            "kernel": "stage_kernel", "avg_launch_ms": avg_launch_ms, "alg_ops_per_launch": ops,
            "alg_ops_per_cell": method_ops_per_cell_stage(F), "kernel_ops_per_cell": kernel_ops_per_cell_stage(F),
            "kernel_ops_frac": kernel_ops_per_cell_stage(F) * cells / (avg_launch_ms * 1e-3) / 1e12 / pk}
    return roof, hbm


def _line(args, world, value, ms_total, dtype, config, extra):
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config}
    line.update(extra)
    return line


def run_ensemble(args, members, dtype, rank, world, barrier):
    """Batched ensemble: every RK stage of all members is one persistent launch over a (member, tile)
    work table; the three launches of a step are replayed from a CUDA graph."""
    import torch
    from paper_1507_08549_gb300 import hydro
    hs = [hydro.Hydro(p, dtype=dtype) for p in members]
    Us = [h.state(p.U0) for h, p in zip(hs, members)]
    cells = sum(p.cells for p in members)
    tune_ms, best = hydro.hydro_batch_autotune(hs, Us, steps=3) if args.autotune else (None, None)
    hydro.hydro_batch_step(hs, Us, args.warmup)
    torch.cuda.synchronize()
    l0 = sum(h.launch_count() for h in hs)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hydro.hydro_batch_step(hs, Us, args.steps)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    launches = sum(h.launch_count() for h in hs) - l0
    F, B = members[0].nfields, (8 if dtype == "f64" else 4)
    roof, roof_hbm = roofline(F, B, cells, ms / (3 * args.steps), (clk or {}).get("sm_mhz"), alu=(dtype == "f32"))
    roof["note"] = "launch time from the whole timed region / (3 x steps): includes packing and graph launch"
    for h in hs:
        h.close()
    if rank == 0:
        sizes = sorted({(p.nx, p.ny) for p in members})
        cfg = {"workload": args.workload, "members": len(members), "cells": cells, "sizes": len(sizes),
               "seed": members[0].seed, "graph": "3 persistent launches per step, replayed from a CUDA graph",
               "autotune": None if best is None else {"best": hydro.batch_trial(best),
                                                      "trials_ms_per_step": [round(float(x), 4) for x in tune_ms]}}
        print(json.dumps(_line(args, world, replica_rate(cells * args.steps, ms * 1e-3, world), ms, dtype, cfg,
                               {"roofline": roof, "roofline_hbm": roof_hbm, "gpu_launches": launches,
                                "clocks": clk})), flush=True)
    return 0


def run_gradient(args, prob, dtype, rank, world, barrier):
    """Gradient configuration: forward run of `steps` steps with checkpoints every 20, then the reverse
    sweep of the discrete adjoint; reports the forward rate and the adjoint / forward time ratio."""
    import torch
    from paper_1507_08549_gb300 import hydro
    h = hydro.Hydro(prob, dtype=dtype)
    U = h.state(prob.U0)
    h.step(U, args.warmup)
    U = h.state(prob.U0)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    h.forward_checkpointed(U, args.steps, 20)
    torch.cuda.synchronize()
    fwd = time.perf_counter() - t0
    # cotangent of the configuration's objective J = sum (m_x^2 + m_y^2) / (2 rho) dx dy at the final state
    rho, mx, my = U[0], U[1], U[2]
    dA = prob.dx * prob.dy
    lam = torch.zeros_like(U)
    lam[0] = -0.5 * (mx * mx + my * my) / (rho * rho) * dA
    lam[1] = mx / rho * dA
    lam[2] = my / rho * dA
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.adjoint_sweep(lam)
    torch.cuda.synchronize()
    adj = time.perf_counter() - t0
    barrier()
    fwd, adj = max_over_ranks(fwd, world), max_over_ranks(adj, world)
    h.close()
    if rank == 0:
        cfg = {"workload": args.workload, "nx": prob.nx, "ny": prob.ny, "checkpoint_every": 20}
        extra = {"adjoint": {"sweep_ms": adj * 1e3, "forward_ms": fwd * 1e3, "adjoint_over_forward": adj / fwd},
                 "e2e": None}
        print(json.dumps(_line(args, world, replica_rate(prob.cells * args.steps, fwd, world), fwd * 1e3, dtype, cfg,
                               extra)),
              flush=True)
    return 0


def _timed(fn, local):
    """Run fn() between CUDA events on the current stream with the clock sampler running; returns
    (ms, clocks, fn's result)."""
    import torch
    clocks = Clocks(local)
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), clocks.stop(), out


def host_link(nbytes: int, local: int):
    """Plain copy-engine rates between pinned host memory and the device for one state's worth of bytes:
    the ceiling of the end-to-end (host-buffer) figure. Best of 3 per direction, CUDA events."""
    import torch
    n = nbytes // 4
    host = torch.empty(n, dtype=torch.float32).pin_memory()
    dev = torch.empty(n, dtype=torch.float32, device="cuda")
    dev.copy_(host, non_blocking=True)
    host.copy_(dev, non_blocking=True)
    best_h2d = best_d2h = float("inf")
    for _ in range(3):
        ms, _, _ = _timed(lambda: dev.copy_(host, non_blocking=True), local)
        best_h2d = min(best_h2d, ms)
        ms, _, _ = _timed(lambda: host.copy_(dev, non_blocking=True), local)
        best_d2h = min(best_d2h, ms)
    del host, dev
    return {"bytes": 4 * n, "h2d_gbs": 4 * n / (best_h2d * 1e-3) / 1e9, "d2h_gbs": 4 * n / (best_d2h * 1e-3) / 1e9,
            "how": "torch copy_ between a pinned host tensor and a device tensor (cudaMemcpyAsync), best of 3"}


def config_records(args, local):
    """Short timed records of the other workload configurations, beside the 8192^2 headline: the plain
    method (128^2 FP64, 100 steps), the (r,z) Rayleigh-Taylor grid (1024 x 2048, FP32 and FP64), the
    64-member ensemble (one persistent launch per stage, CUDA graph) and the 256^2 gradient configuration
    (200 steps, checkpoints every 20, forward and adjoint sweep, FP64 and FP32). Each: cell-updates/s,
    milliseconds per step, the HBM fraction of its algorithmic bytes and the clocks sampled while it ran."""
    import torch
    from paper_1507_08549_gb300 import hydro
    from paper_1507_08549_gb300 import workloads as wl
    out = {}
    peak, _ = _peaks()

    def single(name, prob, dtype, steps, warmup=3):
        h = hydro.Hydro(prob, dtype=dtype)
        U = h.state(prob.U0)
        tune = [round(x, 4) for x in h.autotune(U, steps=2)]
        info = h.tile_info(h.tile_variants()[1])
        h.step(U, warmup)
        ms, clk, _ = _timed(lambda: h.step(U, steps), local)
        h.close()
        B = 8 if dtype == "f64" else 4
        alg = 8 * prob.nfields * B * prob.cells  # bytes per RK3 step
        rec = {"workload": name, "dtype": dtype, "cells": prob.cells, "steps": steps, "ms_per_step": ms / steps,
               "value": prob.cells * steps / (ms * 1e-3), "unit": UNIT,
               "roofline_hbm": {"achieved": alg / (ms / steps * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                                "frac": alg / (ms / steps * 1e-3) / 1e9 / peak},
               "l2": ("state in L2" if prob.nfields * B * prob.cells < 129e6 else "state larger than L2"),
               "tile": info, "autotune_ms_per_step": tune, "clocks": clk}
        return rec

    out["c1_advected_wave_128_f64"] = single("advected_wave_128", wl.advected_wave(128), "f64", 100)
    rt = wl.rayleigh_taylor(1024, 2048)
    out["c2_rayleigh_taylor_1024x2048_f32"] = single("rayleigh_taylor_1024x2048", rt, "f32", 300)
    out["c2_rayleigh_taylor_1024x2048_f64"] = single("rayleigh_taylor_1024x2048", rt, "f64", 3)
    del rt
    # C3: the 64-member ensemble
    members = wl.quadrant_ensemble(64)
    hs = [hydro.Hydro(p, dtype="f32") for p in members]
    Us = [h.state(p.U0) for h, p in zip(hs, members)]
    cells = sum(p.cells for p in members)
    hydro.hydro_batch_step(hs, Us, 3)
    steps = 10
    ms_default, _, _ = _timed(lambda: hydro.hydro_batch_step(hs, Us, steps), local)
    tune_ms, best = hydro.hydro_batch_autotune(hs, Us, steps=3)
    hydro.hydro_batch_step(hs, Us, 1)
    ms, clk, _ = _timed(lambda: hydro.hydro_batch_step(hs, Us, steps), local)
    for h in hs:
        h.close()
    alg = 8 * 4 * 4 * cells
    out["c3_quadrant_ensemble_64_f32"] = {
        "workload": "quadrant_ensemble_64", "dtype": "f32", "members": len(members), "cells": cells, "steps": steps,
        "ms_per_step": ms / steps, "value": cells * steps / (ms * 1e-3), "unit": UNIT,
        "roofline_hbm": {"achieved": alg / (ms / steps * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (ms / steps * 1e-3) / 1e9 / peak},
        "note": "timed region includes each call's packing and unpacking of the 64 caller states", "clocks": clk,
        "default_plan_ms_per_step": ms_default / steps,
        "autotune": {"best": hydro.batch_trial(best), "trials_ms_per_step": {
            f"v{hydro.batch_trial(i)['variant']}_w{hydro.batch_trial(i)['waves']}_{hydro.batch_trial(i)['layout']}":
            round(float(x), 4) for i, x in enumerate(tune_ms)}}}
    del hs, Us, members
    # C4: the gradient configuration
    prob, _ = wl.fourier_modes(256, nsteps=200)
    for dtype in ("f64", "f32"):
        h = hydro.Hydro(prob, dtype=dtype)
        U = h.state(prob.U0)
        h.step(U, 3)
        U = h.state(prob.U0)
        fwd_ms, clk, _ = _timed(lambda: h.forward_checkpointed(U, 200, 20), local)
        rho, mx, my = U[0], U[1], U[2]
        dA = prob.dx * prob.dy
        lam = torch.zeros_like(U)
        lam[0] = -0.5 * (mx * mx + my * my) / (rho * rho) * dA
        lam[1] = mx / rho * dA
        lam[2] = my / rho * dA
        adj_ms, clk2, _ = _timed(lambda: h.adjoint_sweep(lam), local)
        h.close()
        out[f"c4_fourier_256_gradient_{dtype}"] = {
            "workload": "fourier_256_adjoint", "dtype": dtype, "cells": prob.cells, "steps": 200,
            "checkpoint_every": 20, "forward_ms": fwd_ms, "adjoint_sweep_ms": adj_ms,
            "adjoint_over_forward": adj_ms / fwd_ms, "value": prob.cells * 200 / (fwd_ms * 1e-3), "unit": UNIT,
            "clocks": clk, "clocks_adjoint": clk2}
    return out


def run(args):
    import torch
    import torch.distributed as dist
    from paper_1507_08549_gb300 import hydro
    from paper_1507_08549_gb300 import workloads as wl

    rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    prob = workload(args.workload)
    dtype = args.dtype or WORKLOADS[args.workload][1]
    char = args.scheme == "characteristic"
    if char:
        if args.workload in ("quadrant_ensemble_64", "fourier_256_adjoint"):
            raise SystemExit("the characteristic scheme runs single-grid forward workloads")
        prob = prob.with_(scheme=1)
    if args.workload == "quadrant_ensemble_64":
        return run_ensemble(args, prob, dtype, rank, world, barrier)
    if args.workload == "fourier_256_adjoint":
        return run_gradient(args, prob, dtype, rank, world, barrier)
    h = hydro.Hydro(prob, dtype=dtype)
    U = h.state(prob.U0)
    tune = None
    if args.variant is not None:
        h.set_tile_variant(args.variant)
    elif not args.no_autotune:
        # the library's tile autotuner (hydro_autotune) times every variant on this state (left untouched)
        # and keeps the fastest for the timed steps
        tune = [round(x, 4) for x in h.autotune(U, steps=2)]
    n_var, var = h.tile_variants()
    info = h.tile_info(var)
    # warm-up (untimed)
    h.step(U, args.warmup)
    torch.cuda.synchronize()

    def timed_region():
        launches0 = h.launch_count()
        h.profile(True)
        clocks = Clocks(local)
        clocks.start()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        t_sim, _ = h.step(U, args.steps)
        e1.record()
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        nl, sms = h.stage_timing()
        h.profile(False)
        return e0.elapsed_time(e1), clk, t_sim, nl, sms, h.launch_count() - launches0

    ms, clk, t_sim, nlaunch_stage, stage_ms, gpu_launches = timed_region()
    rejected = clocks_rejected(clk)
    if max_over_ranks(1.0 if rejected else 0.0, world) > 0:  # every rank takes the same branch
        ms, clk, t_sim, nlaunch_stage, stage_ms, gpu_launches = timed_region()
        if clk is not None:
            clk["remeasured_after"] = rejected or "another rank's clock record"
    ms = max_over_ranks(ms, world)
    cells = prob.nx * prob.ny
    value = replica_rate(cells * args.steps, ms * 1e-3, world)
    F, B = prob.nfields, (8 if dtype == "f64" else 4)
    traffic = None
    per_cell = stage_traffic_per_cell(f"{info['tile_x']}x{info['tile_y']}")
    if dtype == "f32" and F == 5 and args.workload.startswith("blobs_blast") and per_cell is not None:
        # measured average traffic of a stage launch per cell of this kernel source, times cells
        traffic = per_cell * cells
    roof, roof_hbm = roofline(F, B, cells, stage_ms / max(nlaunch_stage, 1), (clk or {}).get("sm_mhz"),
                              alu=(dtype == "f32" and not char), traffic=None if char else traffic)
    if char:  # two kernels per stage (char_div_kernel, stage_kernel), timed together
        roof["kernel"] = "char_div_kernel + stage_kernel"
    # end to end through the public host-buffer entry: every step copies the state in and out
    if args.quick:
        h.close()
        if rank == 0:
            cfg = {"workload": args.workload, "scheme": args.scheme, "nx": prob.nx, "ny": prob.ny, "nfields": F,
                   "cells": cells, "tile": info, "autotune_ms_per_step": tune}
            print(json.dumps(_line(args, world, value, ms, dtype, cfg, {"roofline": roof, "roofline_hbm": roof_hbm,
                                                                       "gpu_launches": gpu_launches,
                                                                       "clocks": clk})), flush=True)
        return 0
    Uh_pinned = U.cpu().pin_memory().numpy()
    h.step_host(Uh_pinned, 1)
    torch.cuda.synchronize()
    ke = max(1, min(args.steps, args.e2e_steps))
    # three runs of ke one-step calls; the median run is reported (the host link is shared with the rest of
    # the machine, and a single run has shown a 20 % outlier)
    runs = []
    for _ in range(3):
        barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            h.step_host(Uh_pinned, 1)
        runs.append(max_over_ranks(time.perf_counter() - t0, world))
        barrier()
    e2e_s = statistics.median(runs)
    state_bytes = F * B * cells
    e2e = {"value": replica_rate(cells * ke, e2e_s, world), "unit": UNIT, "h2d_bytes_per_step": state_bytes,
           "d2h_bytes_per_step": state_bytes, "steps": ke, "runs_ms_per_step": [round(r / ke * 1e3, 3) for r in runs],
           "how": "median of 3 runs of ke one-step calls with pinned host buffers"}
    del Uh_pinned
    link = host_link(state_bytes, local)
    e2e["host_link"] = link
    # the copies alone bound the end-to-end rate: one state in and one out per step at the plain copy rates
    e2e["copy_bound_value"] = cells / (state_bytes / (link["h2d_gbs"] * 1e9) + state_bytes / (link["d2h_gbs"] * 1e9))
    # FP32 discrete adjoint of one step (frozen dt / alphas of the step it reverses) and the FP64 plain step
    adjoint = None
    if not args.no_adjoint and args.workload == "blobs_blast_8192" and not char:
        h.record(2)
        h.step(U, 1)
        dtl, al = h.get_log(1)
        h.record(0)
        # a seeded non-constant cotangent (a constant one would zero every face adjoint in the first
        # reversed stage and let the line adjoint skip its WENO gradients)
        gen = torch.Generator(device=U.device).manual_seed(wl.DEFAULT_SEED)
        lam = torch.rand(U.shape, generator=gen, device=U.device, dtype=U.dtype) * 2 - 1
        h.adjoint_step(U, lam.clone(), float(dtl[0]), al[0].ravel())  # warm-up (allocates the adjoint buffers)
        torch.cuda.synchronize()
        ka = max(1, args.adjoint_steps)
        lam_k = [lam.clone() for _ in range(ka)]  # adjoint_step overwrites its cotangent in place
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for k in range(ka):
            h.adjoint_step(U, lam_k[k], float(dtl[0]), al[0].ravel())
        a1.record()
        torch.cuda.synchronize()
        adj_ms = a0.elapsed_time(a1) / ka
        adjoint = {"ms_per_step": adj_ms, "dtype": dtype, "steps": ka,
                   "adjoint_over_forward": adj_ms / (ms / args.steps)}
    # level-set reinitialisation of the state's phi, timed once after a warm-up call
    reinit = None
    if args.workload == "blobs_blast_8192":
        h.reinit(U)
        torch.cuda.synchronize()
        r0_, r1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0_.record()
        npts = h.reinit(U)
        r1_.record()
        torch.cuda.synchronize()
        reinit = {"ms": r0_.elapsed_time(r1_), "front_points": npts,
                  "pair_distances_per_s": npts * cells / (r0_.elapsed_time(r1_) * 1e-3)}
    h.close()
    # measured FMA throughput: the cross-check of the derived arithmetic roofline
    alu_probe = None
    if args.workload == "blobs_blast_8192":
        hp = hydro.Hydro(prob.with_(nx=64, ny=64, U0=prob.U0[:, :64, :64].copy()), dtype="f32")
        f32 = hp.fma_probe("f32", 65536)
        f64 = hp.fma_probe("f64", 2048)
        hp.close()
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        alu_probe = {"fp32_fma_per_s": f32, "fp64_fma_per_s": f64,
                     "fp32_derived_fma_per_s": sms * 128 * mhz * 1e6, "fp32_measured_over_derived":
                     f32 / (sms * 128 * mhz * 1e6), "fp64_over_fp32": f64 / f32,
                     "how": "8 independent FMA chains per thread, 8 CTAs of 256 threads per SM (hydro_fma_probe)"}
    characteristic = None
    if args.workload == "blobs_blast_8192" and not char and not args.no_char:
        # the characteristic-wise scheme (Roe-averaged eigenvectors) on the same state, FP32
        hc = hydro.Hydro(prob.with_(scheme=1), dtype=dtype)
        Uc = hc.state(prob.U0)
        hc.step(Uc, 1)
        torch.cuda.synchronize()
        kc = max(1, args.char_steps)
        c0_, c1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0_.record()
        hc.step(Uc, kc)
        c1_.record()
        torch.cuda.synchronize()
        msc = c0_.elapsed_time(c1_) / kc
        characteristic = {"ms_per_step": msc, "value": cells / (msc * 1e-3), "unit": UNIT, "steps": kc,
                          "dtype": dtype, "over_component": msc / (ms / args.steps)}
        hc.close()
        del Uc
    five_stage = None
    if args.workload == "blobs_blast_8192" and not char and not args.no_rk5:
        # the paper's five-stage third-order scheme (five stage launches per step) on the same state
        h5 = hydro.Hydro(prob.with_(rk_stages=5), dtype=dtype)
        U5 = h5.state(prob.U0)
        h5.step(U5, 1)
        torch.cuda.synchronize()
        k5 = max(1, args.rk5_steps)
        q0_, q1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0_.record()
        h5.step(U5, k5)
        q1_.record()
        torch.cuda.synchronize()
        ms5 = q0_.elapsed_time(q1_) / k5
        five_stage = {"ms_per_step": ms5, "value": cells / (ms5 * 1e-3), "unit": "cell-updates/s per 5-stage step",
                      "steps": k5, "dtype": dtype, "stages": 5, "over_rk3_step": ms5 / (ms / args.steps)}
        h5.close()
        del U5
    poisson = poisson_timing(args) if args.workload == "blobs_blast_8192" and not args.no_poisson else None
    configs = config_records(args, local) if args.workload == "blobs_blast_8192" and not args.no_configs else None
    fp64 = None
    if not args.no_fp64 and dtype == "f32" and args.workload == "blobs_blast_8192":
        h64 = hydro.Hydro(prob, dtype="f64")
        U64 = h64.state(prob.U0)
        h64.step(U64, 1)
        torch.cuda.synchronize()
        k64 = max(1, args.fp64_steps)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record()
        h64.step(U64, k64)
        b1.record()
        torch.cuda.synchronize()
        ms64 = b0.elapsed_time(b1) / k64
        fp64 = {"ms_per_step": ms64, "value": cells / (ms64 * 1e-3), "unit": UNIT, "steps": k64,
                "fp64_over_fp32": ms64 / (ms / args.steps)}
        h64.close()
        del U64
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": {"workload": args.workload, "scheme": args.scheme, "nx": prob.nx, "ny": prob.ny, "nfields": F,
                           "cells": cells, "steps_simulated": args.steps, "t_end": t_sim,
                           "l2": (f"state {F * B * cells / 1e9:.2f} GB per copy > 129 MB L2: no flush needed"
                                  if F * B * cells > 129e6 else
                                  f"state {F * B * cells / 1e6:.1f} MB per copy fits in L2: steps back to back,"
                                  " in-L2 rate (not an HBM-bound measurement)"),
                           "tile": info, "autotune_ms_per_step": tune,
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roof, "roofline_hbm": roof_hbm, "e2e": e2e, "gpu_launches": gpu_launches, "clocks": clk,
                "adjoint": adjoint, "fp64_step": fp64, "reinit": reinit,
                "characteristic": characteristic, "five_stage": five_stage, "poisson": poisson, "alu_probe": alu_probe,
                "configs": configs}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(prob, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# FP64 operations of one SOR cell update as the method defines them (each rounded operation one, a
# division one): 4 products and 3 sums of the neighbour terms, 4 pi G rho and its subtraction, the
# division by the diagonal, the relaxation blend (2 products, 1 sum), and the relative change (1
# difference, 1 division) of the stopping test.
SOR_OPS_PER_CELL = 16
# nominal FP64 rate of a GB300, 1.25 TFLOP/s with a fused multiply-add as two: 0.625 T operations/s at
# the 2070 MHz maximum SM clock, one operation per FP64 pipe slot
FP64_OPS_NOMINAL = 0.625e12


def adjoint_timing(args):
    """FP32 discrete adjoint of one step of a blobs + blast state (--workload blobs_blast_<n>): `warmup`
    forward steps, the step to reverse recorded (its dt and alphas frozen), one warm-up adjoint step, then
    `adjoint_steps` timed adjoint steps with a seeded random cotangent, next to `steps` forward steps."""
    import torch
    from paper_1507_08549_gb300 import hydro
    from paper_1507_08549_gb300 import workloads as wl
    if not args.workload.startswith("blobs_blast"):
        raise SystemExit("--only-adjoint times a blobs_blast workload")
    prob = workload(args.workload)
    h = hydro.Hydro(prob, dtype="f32")
    U = h.state(prob.U0)
    h.step(U, args.warmup)
    h.record(2)
    h.step(U, 1)
    dtl, al = h.get_log(1)
    h.record(0)
    gen = torch.Generator(device=U.device).manual_seed(wl.DEFAULT_SEED)
    lam = torch.rand(U.shape, generator=gen, device=U.device, dtype=U.dtype) * 2 - 1
    h.adjoint_step(U, lam.clone(), float(dtl[0]), al[0].ravel())
    ka = max(1, args.adjoint_steps)
    lam_k = [lam.clone() for _ in range(ka)]
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record()
    for k in range(ka):
        h.adjoint_step(U, lam_k[k], float(dtl[0]), al[0].ravel())
    a1.record()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    h.step(U, args.steps)
    f1.record()
    torch.cuda.synchronize()
    h.close()
    adj_ms, fwd_ms = a0.elapsed_time(a1) / ka, f0.elapsed_time(f1) / args.steps
    return {"workload": args.workload, "dtype": "f32", "adjoint_ms_per_step": adj_ms, "forward_ms_per_step": fwd_ms,
            "adjoint_over_forward": adj_ms / fwd_ms, "adjoint_steps": ka, "cotangent": "seeded uniform [-1, 1]"}


def poisson_timing(args):
    """Self-gravity potential of the 1024 x 2048 (r,z) star (hydro_poisson): (a) a fixed number of
    red-black sweeps (tol = 0) from a zero guess, timed with CUDA events after a warm-up solve; (b) a
    solve to the relative-change tolerance 1e-8 from a zero guess, and (c) the same again warm-started
    from (b)'s potential after the density changed by 1e-4 (as between two hydro steps)."""
    import torch
    from paper_1507_08549_gb300 import hydro
    from paper_1507_08549_gb300 import workloads as wl
    prob = wl.self_gravity_star()
    h = hydro.Hydro(prob, dtype="f32")
    U = h.state(prob.U0)
    cells = prob.nx * prob.ny
    omega = 2.0 / (1.0 + math.pi / max(prob.nx, prob.ny))
    k = max(1, args.poisson_sweeps)
    phi = torch.zeros((prob.ny, prob.nx), dtype=torch.float64, device=h.device)
    h.poisson(U, omega=omega, tol=0.0, max_iters=64, phi=phi)  # warm-up: allocation and graph capture
    phi.zero_()
    torch.cuda.synchronize()
    launches0 = h.launch_count()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, n_fixed, mass = h.poisson(U, omega=omega, tol=0.0, max_iters=k, phi=phi)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = h.launch_count() - launches0
    if getattr(args, "quick", False):  # profiling runs: the fixed sweeps only
        clocks.stop()
        h.close()
        return {"workload": prob.name, "cells": cells, "sweeps": n_fixed, "ms": ms, "gpu_launches": launches}
    phi.zero_()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record()
    _, n_cold, _ = h.poisson(U, omega=omega, tol=1e-8, max_iters=200000, phi=phi)
    c1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()  # sampled over the fixed-sweep and the cold solves
    cold_ms = c0.elapsed_time(c1)
    U[0].mul_(1.0 + 1e-4)
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0.record()
    _, n_warm, _ = h.poisson(U, omega=omega, tol=1e-8, max_iters=200000, phi=phi)
    w1.record()
    torch.cuda.synchronize()
    warm_ms = w0.elapsed_time(w1)
    h.close()
    ups = cells * n_fixed / (ms * 1e-3)
    achieved = SOR_OPS_PER_CELL * ups / 1e12
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = FP64_OPS_NOMINAL * mhz / 2070.0 / 1e12
    return {"workload": prob.name, "cells": cells, "omega": omega, "dtype": "f64", "grid_mass": mass,
            "fixed": {"sweeps": n_fixed, "ms": ms, "ms_per_sweep": ms / n_fixed, "cell_updates_per_s": ups,
                      "gpu_launches": launches, "clocks": clk},
            "converged_cold": {"tol": 1e-8, "sweeps": n_cold, "ms": cold_ms},
            "converged_warm": {"tol": 1e-8, "sweeps": n_warm, "ms": warm_ms, "density_change": 1e-4},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP64 ops/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "sor_color_kernel",
                         "peak_kind": f"derived: nominal 1.25 TFLOP/s FP64 (FMA = 2) as {FP64_OPS_NOMINAL / 1e12:.3f} "
                                      f"T ops/s at 2070 MHz, scaled to {mhz:.0f} MHz",
                         "alg_ops_per_cell_update": SOR_OPS_PER_CELL,
                         "l2": f"phi + rho = {cells * 12 / 1e6:.0f} MB stay in the 129 MB L2 across sweeps"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="blobs_blast_8192", choices=sorted(WORKLOADS))
    ap.add_argument("--dtype", default=None, choices=["f32", "f64"])
    ap.add_argument("--autotune", action="store_true", help="ensemble workload: tune the batch plan first")
    ap.add_argument("--no-autotune", action="store_true", help="single grids: keep the default tile variant")
    ap.add_argument("--variant", type=int, default=None, help="tile variant (see hydro_tile_info)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--quick", action="store_true", help="forward timing only (profiling runs)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-poisson", action="store_true")
    ap.add_argument("--scheme", default="component", choices=["component", "characteristic"],
                    help="flux reconstruction of the timed run")
    ap.add_argument("--no-char", action="store_true", help="skip the characteristic-scheme timing")
    ap.add_argument("--char-steps", type=int, default=5)
    ap.add_argument("--no-configs", action="store_true", help="skip the timed records of the other configurations")
    ap.add_argument("--no-rk5", action="store_true", help="skip the five-stage scheme timing")
    ap.add_argument("--rk5-steps", type=int, default=5)
    ap.add_argument("--poisson-sweeps", type=int, default=2048)
    ap.add_argument("--only-poisson", action="store_true",
                    help="time the self-gravity Poisson solve alone and print its JSON (profiling)")
    ap.add_argument("--only-adjoint", action="store_true",
                    help="time the FP32 adjoint step of a blobs + blast workload alone and print its JSON "
                         "(profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    if args.only_poisson:
        print(json.dumps(poisson_timing(args)), flush=True)
        return 0
    if args.only_adjoint:
        print(json.dumps(adjoint_timing(args)), flush=True)
        return 0
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
