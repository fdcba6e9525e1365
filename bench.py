#!/usr/bin/env python3
"""Benchmark of the batched octree hydro step on GB300.

One step = one SSP-RK3 time step of the whole hot path over the workload:
three RK stages (halo gather from the neighbours' interiors, PPM
reconstruction, central-upwind flux, maximum-speed reduction, flux-divergence
update), the time step chosen on the device from the previous step's CFL
speed, and the conservation totals; the mixed path also writes the FP32 shadow
of the state once per step (each stage then writes its output's shadow).  The metric is interior cell-updates per second
(cells x 3 stages / step time).

Workload (default): the largest configuration, a 65536-leaf octree of 8^3
sub-grids (33.5 M interior cells, two n=1.5 polytropes, 656 Zipf batches).
The headline value is the mixed FP32/FP64 path; the all-FP64 path is measured
on the same input and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (under torchrun) runs N independent replicas, one per GPU, and reports
the aggregate; the reference arm times the CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "hydro cell-updates/s (FP64 vs FP32/FP64-mixed batched) at stated error; % HBM roofline"
BYTES_PER_CELL_STAGE = 374.0     # read interior + 6 face slabs (1664 cells) + write interior (512), 88 B per cell
# one RK3 step's stages: stage 1 moves 374 B per cell, stages 2 and 3 also read a
# second FP64-sized array (U0, or the previous increment in the mixed increment form)
BYTES_PER_CELL_RK3_STAGE = (374.0 + 2 * 462.0) / 3.0
# FP64 operations per cell-update of the FP64 stage kernel, counted by ncu's per-opcode instruction
# counters on one stage (beta = 1) of the 4097-leaf reduced binary octree (2,097,664 cells): DADD
# 1,534,302,248, DMUL 1,175,636,249, DFMA 683,163,976 thread instructions
FP64_INST_PER_CELL_STAGE = (1534302248 + 1175636249 + 683163976) / 2097664.0        # 1617.6
FLOPS_PER_CELL_STAGE = (1534302248 + 1175636249 + 2 * 683163976) / 2097664.0       # 1943.3 (an FMA counts 2)
GHOST_BYTES_PER_CELL = 396.0     # ghost fill: read + write 1152 face-slab cells per 512 interior cells
SHADOW_BYTES_PER_CELL = 137.5    # FP32 shadow: read 88 B of FP64 interior, write 44 B + 5.5 B of restriction
TAU_RESYNC_BYTES_PER_CELL = 56.0  # tracer reset: read rho, s, E, tau (48 B), write tau (8 B)
# FP64 peak from the unit count: 152 SMs x 2 FP64 instructions per clock x 2.07 GHz (ncu on the counted
# launch: the FP64 pipe busy 79 % of the active cycles at 1.56 instructions per clock per SM, i.e. about 1.98
# per clock at 100 %); an FMA counts 2 flops
FP64_PEAK_INST = 152 * 2 * 2.070e9
FP64_PEAK_TFLOPS = 2 * FP64_PEAK_INST / 1e12
# FP64 operations per cell-update of one stage of the 3D reconstruction with Simpson face quadrature,
# the plain evaluation of the reading (every operation as written, branches taken per value): ncu's
# per-opcode counters on the kernels' plain form (recon3d_faces + recon3d_flux + recon3d_update, one
# stage on the 64^3 lognormal box, 262,144 cells): DADD 1,542,778,255, DMUL 1,342,567,247, DFMA 760,421,186
RECON3D_FP64_INST_PER_CELL = (1542778255 + 1342567247 + 760421186) / 262144.0      # 13907.5
RECON3D_FLOPS_PER_CELL = (1542778255 + 1342567247 + 2 * 760421186) / 262144.0     # 16808.3
# DRAM bytes (read + write) per cell-update of the mixed stage kernel from one ncu capture
# (average of the three RK3 stage launches), valid only for the kernel sources it was taken on
# (STAGE_SOURCES, hashed in that order).
STAGE_TRAFFIC = {"sha256_prefix": "61593a21ff5defa8", "bytes_per_cell": 302.4,
                 "source": "ncu capture of the three RK3 stage launches on the 4097-leaf reduced binary octree "
                           "(average), scaled by cells"}


STAGE_SOURCES = ("hydro_stage.cu", "hydro_scheme.cuh", "hydro_cw84.cuh", "hydro_reflux.cuh", "hydro_fp.cuh",
                 "hydro_internal.cuh")


def stage_source_sha():
    """sha256 of the stage kernel's sources (the .cu file and the headers it includes, in that order)."""
    import hashlib
    h = hashlib.sha256()
    for name in STAGE_SOURCES:
        with open(os.path.join(ROOT, "paper_2210_06437_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def stage_traffic_bytes(cells):
    """Measured DRAM traffic of one mixed stage launch, or None if the kernel
    source changed since the counters were taken."""
    if not stage_source_sha().startswith(STAGE_TRAFFIC["sha256_prefix"]):
        return None
    return STAGE_TRAFFIC["bytes_per_cell"] * cells


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--config", type=int, default=5, help="workload configuration 1..5")
    p.add_argument("--skip-e2e", action="store_true")
    p.add_argument("--skip-fp64", action="store_true")
    p.add_argument("--skip-cpu", action="store_true")
    p.add_argument("--stage-only", choices=["mixed", "fp64"], default=None,
                   help="profiling case: one RK3 step (mixed: the three stage launches of the increment form with "
                        "their correction passes) or one FP64 stage (beta = 1) on --config with default launch "
                        "parameters, then exit; prints no benchmark line")
    p.add_argument("--cw84", type=int, default=0, help="profiling case: CW84 extensions (HYDRO_PARAM_CW84 bits)")
    p.add_argument("--fused", type=int, default=0, help="profiling case: the one-launch RK3 step (1)")
    p.add_argument("--recon3d", type=int, default=0,
                   help="profiling case (FP64, a grid of one level): the 3D reconstruction with Simpson face "
                        "quadrature (1)")
    p.add_argument("--skip-recon3d", action="store_true")
    p.add_argument("--sweep", action="store_true",
                   help="per-configuration table (one JSON line per configuration and precision, errors against "
                        "the oracle, oracle timings); not the benchmark line")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower().startswith("active")})
        busy = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": float(np.median(busy)) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(dist, x: float, device) -> float:
    """Largest value of x over all ranks (the step time of the slowest replica)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(cells_per_rank: int, stages: int, world: int, seconds_max: float) -> float:
    """Whole-job cell-updates/s: every rank advances its own replica of the
    workload, and the job takes as long as the slowest rank."""
    return cells_per_rank * stages * world / seconds_max


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_rate(w, U, out, target_s=10.0, seed=0):
    """Oracle cell-updates/s of one RK stage on a bounded random sample of the
    workload's sub-grids (all host threads); the sample grows until one stage
    takes at least target_s.  `out` receives only the sampled interiors."""
    import oracle
    o = oracle.Oracle(w.grid)
    rng = np.random.default_rng(seed)
    n = 32
    while True:
        ids = np.sort(rng.choice(w.grid.n, min(n, w.grid.n), replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        o.stage(U, 1e-6, Uout=out, ids=ids, batch_all=True)
        t = time.perf_counter() - t0
        if t >= target_s or n >= w.grid.n:
            break
        n = min(w.grid.n, int(n * max(2.0, min(8.0, target_s / max(t, 1e-3)))))
    return len(ids) * 512 / t, len(ids), t


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    from paper_2210_06437_gb300 import workloads as W
    oracle.build()
    w = W.config(args.config)
    U = w.state()
    o = oracle.Oracle(w.grid)
    o.fill_ghosts(U)
    # bounded sample: each "step" is three oracle stages on the same sampled sub-grids
    out = np.empty_like(U)
    rate, nsamp, t1 = oracle_rate(w, U, out, target_s=3.0)
    ids = np.sort(np.random.default_rng(1).choice(w.grid.n, nsamp, replace=False)).astype(np.int32)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for beta in (1.0, 0.25, 2.0 / 3.0):
            o.stage(U, 1e-6, U0=U, beta=beta, Uout=out, ids=ids, batch_all=True)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    tstep = float(np.mean(times))
    value = nsamp * 512 * 3 / tstep
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tstep * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "subgrids": w.grid.n, "cells": w.cells},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                             "sample": "3 oracle RK stages per step on %d of %d sub-grids of %s, OpenMP over "
                                       "sub-grids" % (nsamp, w.grid.n, w.name)},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# per-configuration sweep
# ---------------------------------------------------------------------------

def field_errors(x, r, gamma=5.0 / 3.0):
    """Field-maximum error of interior cells (reported beside the per-cell
    metric): max|x_f - r_f| / S_f, S_f = max|r_f|, and for the three momenta
    the momentum-density scale max(|s|, rho c) over the field."""
    sl = (slice(None), slice(None), slice(3, 11), slice(3, 11), slice(3, 11))
    xi, ri = x[sl], r[sl]
    d = np.abs(xi - ri).max(axis=(0, 2, 3, 4))
    S = np.abs(ri).max(axis=(0, 2, 3, 4))
    rho = ri[:, 0]
    s2 = ri[:, 1] ** 2 + ri[:, 2] ** 2 + ri[:, 3] ** 2
    p = (gamma - 1.0) * np.maximum(ri[:, 4] - 0.5 * s2 / rho, 0.0)
    S[1:4] = max(np.sqrt(s2).max(), np.sqrt(gamma * rho * p).max())
    return np.where(S > 0, d / np.where(S > 0, S, 1.0), np.where(d == 0, 0.0, np.inf))


def run_sweep(args):
    """Every workload configuration: one stage and one SSP-RK3 step of each
    precision against the oracle on the same input (the error metric of the
    parity tests), the RK3 step rate of the multi-step graph, and the oracle's
    own rates (all host threads on the whole grid; one thread on a sample)."""
    import torch
    import oracle
    from paper_2210_06437_gb300 import build, hydro as HY
    from paper_2210_06437_gb300 import workloads as W
    from tests import r12 as R
    torch.cuda.set_device(0)
    build.build()
    oracle.build()
    hbm, _ = peaks()
    stream = torch.cuda.current_stream()
    for cfg in (1, 2, 3, 4, 5):
        w = W.config(cfg)
        U = w.state()
        o = oracle.Oracle(w.grid)
        o.fill_ghosts(U)
        _, ms0, _ = o.stage(U, 0.0)
        dt = 0.4 / ms0[1]
        ref1 = np.empty_like(U)   # interiors written by the stage (allocated outside the timing)
        t0 = time.perf_counter()
        o.stage(U, dt, Uout=ref1)
        t_o_stage = time.perf_counter() - t0
        t0 = time.perf_counter()
        ref3, _, _ = o.rk3_step(U, dt)   # as it stands: its stage copies and ghost fills included
        t_o_rk3 = time.perf_counter() - t0
        ids1 = np.sort(np.random.default_rng(cfg).choice(w.grid.n, min(w.grid.n, 64), replace=False)).astype(np.int32)
        tmp = np.empty_like(U)
        t0 = time.perf_counter()
        o.stage(U, dt, Uout=tmp, ids=ids1, nthreads=1, batch_all=True)
        t_o_1 = time.perf_counter() - t0
        del tmp
        row = {"config": cfg, "workload": w.name, "subgrids": w.grid.n, "cells": w.cells,
               "oracle": {"stage_rate_all_threads": w.cells / t_o_stage, "rk3_step_s_all_threads": t_o_rk3,
                          "threads": os.cpu_count(), "stage_rate_1_thread": len(ids1) * 512 / t_o_1,
                          "sample_1_thread": "%d sub-grids" % len(ids1)}}
        ids = torch.as_tensor(w.batches.ids, device="cuda")
        offs = w.batches.offsets
        for prec in ("mixed", "fp64"):
            g = HY.HydroGrid(w.grid, precision=prec)
            Ud = torch.from_numpy(U).cuda()
            out = Ud.clone()
            g.step(Ud, dt, U_out=out, ids=ids, batch_offsets=offs)
            x1 = out.cpu().numpy()
            err1, r1, m1 = field_errors(x1, ref1), R.r12(x1, ref1), R.momentum_scaled(x1, ref1)
            del x1
            V = Ud.clone()
            s1, s2 = torch.empty_like(Ud), torch.empty_like(Ud)
            g.rk3_step(V, dt, s1, s2, ids=ids, batch_offsets=offs)
            g.fill_ghosts(V)
            x3 = V.cpu().numpy()
            err3, r3, m3 = field_errors(x3, ref3), R.r12(x3, ref3), R.momentum_scaled(x3, ref3)
            del x3
            del out
            k = 5 if prec == "mixed" else 2
            msd = torch.zeros(2, dtype=torch.float64, device="cuda")
            g.step(V, 0.0, U_out=s1, ids=ids, batch_offsets=offs, max_speed=msd)
            g.rk3_run_prepare(V, 0.4, s1, s2, msd, k, ids=ids, batch_offsets=offs)
            g.rk3_run_cfl(V, 0.4, s1, s2, msd, k, ids=ids, batch_offsets=offs)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.rk3_run_cfl(V, 0.4, s1, s2, msd, k, ids=ids, batch_offsets=offs)
            e1.record(stream)
            torch.cuda.synchronize()
            g.sync()
            t_step = e0.elapsed_time(e1) / 1e3 / k
            g.close()
            del Ud, V, s1, s2
            torch.cuda.empty_cache()
            row[prec] = {"rk3_step_ms": t_step * 1e3, "cell_updates_per_s": w.cells * 3 / t_step,
                         "hbm_frac_of_measured": BYTES_PER_CELL_RK3_STAGE * w.cells * 3 / t_step / 1e9 / hbm,
                         "r12_one_stage": r1["err"].tolist(), "r12_rk3_step": r3["err"].tolist(),
                         "momentum_rhoc_one_stage": m1.tolist(), "momentum_rhoc_rk3_step": m3.tolist(),
                         "err_field_max_one_stage": float(err1.max()), "err_field_max_rk3_step": float(err3.max()),
                         "tolerance": 1e-5 if prec == "mixed" else 1e-12}
        row["mixed_speedup_vs_fp64"] = row["fp64"]["rk3_step_ms"] / row["mixed"]["rk3_step_ms"]
        print(json.dumps(row), flush=True)
    return 0


def run_stage_only(args):
    """A small, fixed launch sequence for ncu (no tuner, no timing)."""
    import torch
    from paper_2210_06437_gb300 import build, hydro as HY
    from paper_2210_06437_gb300 import workloads as W
    build.build()
    w = W.config(args.config)
    U = torch.from_numpy(w.state()).cuda()
    ids = torch.as_tensor(w.batches.ids, device="cuda")
    g = HY.HydroGrid(w.grid, precision=args.stage_only)
    g.set_param(HY.PARAM_CW84, args.cw84)
    g.set_param(HY.PARAM_FUSED_RK3, args.fused)
    g.set_param(HY.PARAM_RECON3D, args.recon3d)
    ms = torch.zeros(2, dtype=torch.float64, device="cuda")
    s1 = torch.empty_like(U)
    g.step(U, 0.0, U_out=s1, ids=ids, batch_offsets=w.batches.offsets, max_speed=ms)
    dt = 0.4 / float(ms[1])
    if args.stage_only == "mixed" or args.fused:
        g.rk3_step(U, dt, s1, torch.empty_like(U), ids=ids, batch_offsets=w.batches.offsets)
    else:
        g.step(U, dt, U_out=s1, ids=ids, batch_offsets=w.batches.offsets)
    g.sync()
    g.close()
    print("stage-only %s config %d: %d sub-grids (cw84 %d, one-launch %d, recon3d %d)"
          % (args.stage_only, args.config, w.grid.n, args.cw84, args.fused, args.recon3d))
    return 0


def run_recon3d(dev, stream, steps, warmup):
    """One Shu-Osher stage with the 3D reconstruction and Simpson face
    quadrature (three kernels; FP64, and mixed precision) on the periodic
    128^3 box of one level, timed with CUDA events over `steps` stages after
    `warmup`, beside the face-centre stage (hydro_step: the mixed one with its
    shadow pass) of each precision on the same state.  Returns
    (workload, {form: (s per stage, launches per stage)})."""
    import torch
    from paper_2210_06437_gb300 import hydro as HY
    from paper_2210_06437_gb300 import workloads as W
    w = W.config(7)
    U = torch.from_numpy(w.state()).to(dev)
    out = torch.empty_like(U)
    ms = torch.zeros(2, dtype=torch.float64, device=dev)
    res = {}
    for form in ("simpson", "simpson_mixed", "face_centre", "face_centre_mixed"):
        g = HY.HydroGrid(w.grid, precision="mixed" if form.endswith("mixed") else "fp64")
        g.set_param(HY.PARAM_RECON3D, 0 if form.startswith("face_centre") else 1)
        g.step(U, 0.0, U_out=out, max_speed=ms)
        dt = 0.4 / float(ms[1])
        for _ in range(warmup):
            g.step(U, dt, U_out=out, max_speed=ms)
        torch.cuda.synchronize()
        l0 = g.launches
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            g.step(U, dt, U_out=out, max_speed=ms)
        b.record(stream)
        torch.cuda.synchronize()
        res[form] = (a.elapsed_time(b) / 1e3 / steps, (g.launches - l0) / steps)
        g.sync()
        g.close()
    return w, res


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.stage_only:
        return run_stage_only(args)
    import torch
    rank, world, local = dist_info()
    pg = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        pg = dist
    else:
        torch.cuda.set_device(0)
    from paper_2210_06437_gb300 import build, hydro as HY
    from paper_2210_06437_gb300 import workloads as W
    if rank == 0 or world == 1:
        build.build()
    if pg:
        pg.barrier()
    build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    w = W.config(args.config)
    U_host = w.state()
    cells = w.cells
    hbm, hbm_src = peaks()

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    def ranks_max(x):
        return max_over_ranks(pg, x, dev)

    U = torch.from_numpy(U_host).to(dev)
    s1, s2 = torch.empty_like(U), torch.empty_like(U)
    ids = torch.as_tensor(w.batches.ids, device=dev)
    offs = w.batches.offsets
    stream = torch.cuda.current_stream()
    results = {}

    from paper_2210_06437_gb300 import tune as TU

    def run_precision(prec, sampler):
        g = HY.HydroGrid(w.grid, precision=prec)
        U.copy_(torch.from_numpy(U_host))
        g.fill_ghosts(U)
        tuned = TU.tune(g, U, s1, s2, ids=ids, batch_offsets=offs)   # launch shapes, outside the timed region
        # the tuner's best RK3 step time of each form (three launches, one launch), from its table
        forms = {}
        entry = TU.load_cache().get(TU.cache_key(torch.cuda.get_device_name(), prec, w.grid.n), {})
        for c, t in entry.get("table", []):
            if t is not None and "fused_rk3" in c:
                k = "one_launch_ms" if c["fused_rk3"] else "three_launches_ms"
                forms[k] = min(forms.get(k, t), t)
        ms = torch.zeros(2, dtype=torch.float64, device=dev)
        g.step(U, 0.0, U_out=s1, ids=ids, batch_offsets=offs, max_speed=ms)   # dry stage: first CFL speed
        tots = torch.empty((max(args.steps, args.warmup), 11), dtype=torch.float64, device=dev)
        # W warm-up steps, then the K timed steps in one graph launch (each step:
        # device CFL dt, three stages, totals of the new state)
        g.rk3_run_cfl(U, 0.4, s1, s2, ms, args.warmup, ids=ids, batch_offsets=offs, totals=tots)
        g.rk3_run_prepare(U, 0.4, s1, s2, ms, args.steps, ids=ids, batch_offsets=offs, totals=tots)
        g.sync()
        barrier()
        if sampler:
            sampler.start()
        l0 = g.launches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.rk3_run_cfl(U, 0.4, s1, s2, ms, args.steps, ids=ids, batch_offsets=offs, totals=tots)
        e1.record(stream)
        tot = tots[args.steps - 1]
        barrier()
        clocks = sampler.stop() if sampler else None
        launches = g.launches - l0
        g.sync()
        t_step = ranks_max(e0.elapsed_time(e1) / 1e3 / args.steps)
        # per-kernel timing for the roofline: stage (beta = 1), ghost fill, totals
        reps = 3

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / 1e3 / reps

        ms2 = torch.zeros(2, dtype=torch.float64, device=dev)
        t_shadow = 0.0
        if prec == "mixed":
            # one Shu-Osher stage (hydro_step_shadowed, beta = 1) and the shadow kernel alone
            S_in, S_out = g.shadow(U), g.empty_shadow()
            t_single = timed(lambda: g.step_shadowed(U, S_in, 1e-9, U_out=s1, S_out=S_out, ids=ids,
                                                     batch_offsets=offs, max_speed=ms2))
            t_shadow = timed(lambda: g.shadow(U, S_in))
            del S_in, S_out
        else:
            t_single = timed(lambda: g.step(U, 1e-9, U_out=s1, ids=ids, batch_offsets=offs, max_speed=ms2))
        # the stage kernel as the RK3 graph launches it: K steps without totals,
        # minus the one shadow pass, over the 3K stage launches (the dt kernels
        # take microseconds; each stage's flux-correction pass is counted in)
        U_save = U.clone()
        g.rk3_run_prepare(U, 0.4, s1, s2, ms, args.steps, ids=ids, batch_offsets=offs)
        t_run = timed(lambda: g.rk3_run_cfl(U, 0.4, s1, s2, ms, args.steps, ids=ids, batch_offsets=offs))
        U.copy_(U_save)
        del U_save
        t_stage = (t_run - t_shadow) / (3 * args.steps)
        t_ghost = timed(lambda: g.fill_ghosts(s1))
        t_tot = timed(lambda: g.totals(U, out=tot))
        # the optional dual-energy tracer reset, standalone (not part of the
        # timed step); it leaves U's tracer reset, and U is not read again
        t_resync = timed(lambda: g.tau_resync(U)) if prec == "mixed" else 0.0
        g.sync()
        g.close()
        return dict(forms=forms, t_step=t_step, clocks=clocks, launches=launches, t_stage=t_stage, t_single=t_single,
                    t_ghost=t_ghost, t_tot=t_tot, t_shadow=t_shadow, t_resync=t_resync, totals=tot.cpu().numpy(),
                    tuned=tuned)

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[local] if vis and len(vis.split(",")) > local else str(local)
    results["mixed"] = run_precision("mixed", ClockSampler(smi_index) if rank == 0 else None)
    if not args.skip_fp64:
        results["fp64"] = run_precision("fp64", None)
    if not args.skip_recon3d and world == 1:
        results["recon3d"] = run_recon3d(dev, stream, args.steps, args.warmup)

    # end-to-end through the public API with host buffers (mixed path): the
    # state lives on the host as packed interiors (pinned) and every step
    # uploads it, advances it one RK3 step with its totals, and downloads it
    e2e = None
    if not args.skip_e2e:
        g = HY.HydroGrid(w.grid, precision="mixed")
        n = w.grid.n
        Ph = g.empty_interiors(pin_memory=True)
        Ph.copy_(torch.from_numpy(np.ascontiguousarray(U_host[:, :, 3:11, 3:11, 3:11]).reshape(n, 11, 512)))
        Pd = g.empty_interiors()
        ms = torch.zeros(2, dtype=torch.float64, device=dev)
        tot = torch.empty(11, dtype=torch.float64, device=dev)
        toth = torch.empty(11, dtype=torch.float64, pin_memory=True)
        g.upload(Ph, U, Pd)
        g.step(U, 0.0, U_out=s1, ids=ids, batch_offsets=offs, max_speed=ms)   # first CFL speed
        # copies in 8 chunks, one stream each: chunk k of a step's download and
        # chunk k of the next step's upload follow each other on stream k, so the
        # two directions of the host link overlap; each chunk is unpacked on its
        # stream as soon as it has arrived and packed on its stream before its
        # download, so those passes overlap the other chunks' copies; the compute
        # stream waits for every unpacked chunk
        n_chunks = 8
        bounds = [(n * c // n_chunks, n * (c + 1) // n_chunks) for c in range(n_chunks)]
        cstreams = [torch.cuda.Stream() for _ in range(n_chunks)]
        for cs in cstreams:
            cs.wait_stream(stream)

        def e2e_step():
            ev_up = []
            for (a_, b_), cs in zip(bounds, cstreams):
                with torch.cuda.stream(cs):
                    Pd[a_:b_].copy_(Ph[a_:b_], non_blocking=True)
                    g.unpack(Pd, U, stream=cs, first=a_, count=b_ - a_)
                    ev = torch.cuda.Event()
                    ev.record(cs)
                    ev_up.append(ev)
            for ev in ev_up:
                stream.wait_event(ev)
            g.rk3_step_cfl(U, 0.4, s1, s2, ms, ids=ids, batch_offsets=offs)
            g.totals(U, out=tot)
            toth.copy_(tot, non_blocking=True)
            ev_done = torch.cuda.Event()
            ev_done.record(stream)
            for (a_, b_), cs in zip(bounds, cstreams):
                cs.wait_event(ev_done)
                with torch.cuda.stream(cs):
                    g.pack(U, Pd, stream=cs, first=a_, count=b_ - a_)
                    Ph[a_:b_].copy_(Pd[a_:b_], non_blocking=True)

        def join():
            for cs in cstreams:
                stream.wait_stream(cs)
        for _ in range(max(1, min(args.warmup, 2))):
            e2e_step()
        join()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for cs in cstreams:
            cs.wait_stream(stream)
        for _ in range(args.steps):
            e2e_step()
        join()
        e1.record(stream)
        barrier()
        g.sync()
        t_e2e = ranks_max(e0.elapsed_time(e1) / 1e3 / args.steps)
        nbytes = Pd.numel() * 8
        e2e = {"value": aggregate_rate(cells, 3, world, t_e2e), "unit": "cell-updates/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes + 88, "ms_per_step": t_e2e * 1e3,
               "api": "every step: pinned host packed interiors -> device in 8 chunks on 8 streams, each "
                      "unpacked on arrival (hydro_unpack_interiors_range) + rk3_step_cfl + totals + per-chunk "
                      "pack (hydro_pack_interiors_range) -> pinned host (same chunks; a step's download overlaps "
                      "the next step's upload on the full-duplex host link)"}
        g.close()
        del Ph, Pd

    # CPU oracle baseline on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if not args.skip_cpu and rank == 0 and world == 1:
        import oracle
        oracle.build()
        Uc = U_host
        oracle.Oracle(w.grid).fill_ghosts(Uc)
        rate, nsamp, t = oracle_rate(w, Uc, np.empty_like(Uc), target_s=10.0)
        cpu = {"value": rate, "unit": "cell-updates/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "one oracle RK stage on %d randomly sampled of %d sub-grids of %s (%.1f s, OpenMP over "
                         "sub-grids, all host threads)" % (nsamp, w.grid.n, w.name, t)}

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0
    r = results["mixed"]
    value = aggregate_rate(cells, 3, world, r["t_step"])
    t_st = r["t_stage"]
    ach = BYTES_PER_CELL_RK3_STAGE * cells / t_st / 1e9
    traffic = stage_traffic_bytes(cells)
    roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": traffic,
            "traffic_source": STAGE_TRAFFIC["source"] if traffic else "kernel changed since the last capture",
            "kernel": ("rk3_kernel<float>, the one launch of each mixed SSP-RK3 step (three stages and their "
                       "coarse-fine corrections), a third of its time per stage"
                       if r["tuned"].get("fused_rk3") else
                       "stage_kernel<float>, the 3 stage launches of the mixed SSP-RK3 graph (increment form), "
                       "average; each launch's time includes the coarse-fine flux-correction pass that follows it "
                       "(reflux_kernel, about 4 % of it)"), "peak_source": hbm_src,
            "bytes_per_cell_update": BYTES_PER_CELL_RK3_STAGE, "launch_ms": t_st * 1e3}
    kernels = {
        "stage_mixed_ms": t_st * 1e3, "stage_mixed_single_beta1_ms": r["t_single"] * 1e3,
        "shadow_ms": r["t_shadow"] * 1e3, "ghost_fill_ms": r["t_ghost"] * 1e3,
        "totals_ms": r["t_tot"] * 1e3, "shadow_gbs": SHADOW_BYTES_PER_CELL * cells / r["t_shadow"] / 1e9,
        "ghost_fill_gbs": GHOST_BYTES_PER_CELL * cells / r["t_ghost"] / 1e9,
        "stage_share_of_step": 3 * t_st / r["t_step"], "totals_share_of_step": r["t_tot"] / r["t_step"],
        "tau_resync_ms": r["t_resync"] * 1e3,
        "tau_resync_gbs": TAU_RESYNC_BYTES_PER_CELL * cells / r["t_resync"] / 1e9 if r["t_resync"] > 0 else None,
        "note": "the stage kernel gathers halos from neighbour interiors; the ghost-fill kernel and the optional "
                "dual-energy tracer reset are not part of the step (timed standalone for reference)"}
    line = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["t_step"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "%s (config %d): %s" % (w.name, w.index, w.description), "subgrids": w.grid.n,
                       "cells": cells, "batches": len(offs) - 1, "precision": "mixed",
                       "step": "SSP-RK3 (3 stages with fused halo gather) + totals, device-side CFL dt; the K timed "
                               "steps run as one hydro_rk3_run_cfl graph launch (FP32 shadow written once, then "
                               "by each step's last stage)",
                       "l2": "inputs larger than L2 (%.1f GB state)" % (U.numel() * 8 / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "tuned": r["tuned"],
                       "rk3_forms_tuner_ms": r["forms"]},
            "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": r["launches"], "clocks": r["clocks"]}
    if "fp64" in results:
        f = results["fp64"]
        fl = FLOPS_PER_CELL_STAGE * cells / f["t_stage"] / 1e12  # average of the RK3 graph's stage launches
        inst = FP64_INST_PER_CELL_STAGE * cells / f["t_stage"]
        line["fp64"] = {"value": aggregate_rate(cells, 3, world, f["t_step"]), "ms_per_step": f["t_step"] * 1e3,
                        "rk3_forms_tuner_ms": f["forms"],
                        "roofline": {"bound": "alu", "achieved": fl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                     "frac": fl / FP64_PEAK_TFLOPS, "traffic": None,
                                     "inst_frac": inst / FP64_PEAK_INST,
                                     "counts": "FP64 operations per cell-update counted by ncu (DADD + DMUL + DFMA "
                                               "= %.1f instructions, %.1f flops)" % (FP64_INST_PER_CELL_STAGE,
                                                                                     FLOPS_PER_CELL_STAGE),
                                     "peak_source": "unit count: 152 SMs x 2 FP64 instructions/clk x 2.07 GHz",
                                     "kernel": "rk3_kernel<double> (a third of each step's launch)"
                                               if f["tuned"].get("fused_rk3") else "stage_kernel<double>",
                                     "launch_ms": f["t_stage"] * 1e3,
                                     "hbm_frac": BYTES_PER_CELL_RK3_STAGE * cells / f["t_stage"] / 1e9 / hbm},
                        "gpu_launches": f["launches"]}
        line["mixed_speedup_vs_fp64"] = f["t_step"] / r["t_step"]
    if "recon3d" in results:
        w3, t3 = results["recon3d"]
        t_s, n_l = t3["simpson"]
        counted = RECON3D_FP64_INST_PER_CELL is not None
        inst3 = RECON3D_FP64_INST_PER_CELL * w3.cells / t_s if counted else None
        fl3 = RECON3D_FLOPS_PER_CELL * w3.cells / t_s / 1e12 if counted else None
        line["recon3d"] = {
            "workload": "%s (config %d): %s" % (w3.name, w3.index, w3.description),
            "value": w3.cells / t_s, "unit": "cell-updates/s", "ms_per_stage": t_s * 1e3,
            "launches_per_stage": n_l, "face_centre_fp64_stage_ms": t3["face_centre"][0] * 1e3,
            "cost_vs_face_centre": t_s / t3["face_centre"][0],
            "mixed": {"ms_per_stage": t3["simpson_mixed"][0] * 1e3, "value": w3.cells / t3["simpson_mixed"][0],
                      "speedup_vs_fp64": t_s / t3["simpson_mixed"][0],
                      "face_centre_mixed_stage_ms": t3["face_centre_mixed"][0] * 1e3,
                      "cost_vs_face_centre": t3["simpson_mixed"][0] / t3["face_centre_mixed"][0],
                      "note": "FP32 reconstruction, transverse parabolas, point fluxes and Simpson sums; FP64 "
                              "update"},
            "l2": "inputs larger than L2 (1.0 GB state, 2.6 GB scratch)",
            "roofline": {"bound": "alu", "achieved": fl3, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": fl3 / FP64_PEAK_TFLOPS if counted else None, "traffic": None,
                         "inst_frac": inst3 / FP64_PEAK_INST if counted else None,
                         "counts": ("FP64 operations per cell-update of the plain evaluation, counted by ncu on "
                                    "the three kernels' plain form (DADD + DMUL + DFMA = %.1f instructions, %.1f "
                                    "flops)" % (RECON3D_FP64_INST_PER_CELL, RECON3D_FLOPS_PER_CELL))
                                   if counted else "not counted for this source",
                         "peak_source": "unit count: 152 SMs x 2 FP64 instructions/clk x 2.07 GHz",
                         "kernel": "recon3d_faces + recon3d_flux + recon3d_update (one FP64 stage)"}}
    print(json.dumps(line))
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
