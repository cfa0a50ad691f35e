#!/usr/bin/env python3
"""Throughput benchmark of the SBP-SAT FDTD leapfrog on GB300.

Workload (default): the 512^3 mixed-faces block (h = 1 mm, PMC SAT on the x
faces, PEC SAT on the y faces, absorbing SAT on the z faces, four seeded
dielectric spheres with eps_r in [2, 8], Gaussian sheet source on Ey, one
probe, 0.95 CFL), FP32.  One "step" = one leapfrog time step (H and E
half-steps, closure rows, SAT penalties, source, probe) over the whole grid.
Metric: Gcell-updates/s = cells * steps / time.  The working set (~7 GB) is
far larger than L2, so no flush is needed between steps.

The same line carries the serving stream (512 requests of 32..192 cells per
axis, 500..4000 steps) run to completion three ways: one grid per launch
sequence (the plain FP32 path), the continuous-batching server with every
request submitted at once, and the server under Poisson arrivals (p50/p99
latency); see `serving`.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 it is launched under torchrun; every rank advances its own replica
of the grid (the path has no data-path exchange: replicas only, weak
scaling) and rank 0 prints the JSON line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_H = 36.0      # per cell: read E (3) + H (3), write H (3), FP32
BYTES_E = 40.0      # per cell: read H (3) + E (3) + eps_r (1), write E (3), FP32
BYTES_FUSED = 52.0  # per cell: read E (3) + H (3) + eps_r (1), write H (3) + E (3), FP32
# FP16 field storage: the six fields move 2 bytes per value, eps_r stays FP32
BYTES16 = {"h_update": 18.0, "e_update": 24.0, "band_h": 18.0, "band_e": 24.0, "fused_interior": 28.0}
HBM_NOMINAL_GBS = 7900.0   # GB300 HBM3e nominal bandwidth, context beside the measured copy peak


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--N", type=int, default=512, help="cells per axis of the block workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", choices=["dielectric", "mixed", "serve", "twoblock", "cavity"], default="mixed",
                    help="mixed: the N^3 block with PMC x, PEC y, absorbing z faces and four dielectric "
                         "spheres (default); dielectric: the N^3 dielectric cube; serve: the request stream alone; "
                         "twoblock: two 192x192x96 blocks joined by the interface SAT; cavity: the 20x16x12 PEC "
                         "cavity in FP64")
    ap.add_argument("--no-serve", action="store_true", help="leave the serving stream out of the line")
    ap.add_argument("--precision", choices=["fp32", "fp16"], default="fp32",
                    help="fp16: FP32 arithmetic with FP16 field storage")
    ap.add_argument("--requests", type=int, default=512, help="serving workload: number of requests")
    ap.add_argument("--rho", type=float, default=0.9, help="serving workload: offered load / plain throughput")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default z-block depth")
    ap.add_argument("--scheme", choices=["sbp", "fdtd"], default="sbp",
                    help="fdtd: the plain Yee comparator on the same grid and kernels (PEC workloads)")
    ap.add_argument("--slots", type=int, default=32)
    ap.add_argument("--budget-gib", type=float, default=8.0)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle samples (every 100 ms) around the timed region.

    A short timed region can fall between two samples, so `wait_for_sample`
    holds the caller until a sample newer than a given time exists: called
    before the region starts and after it ends, it brackets the region with
    the nearest sample on each side.  `summary(t0, t1)` reports the samples in
    [t0, t1] plus those two brackets."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []          # (host time, fields)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def wait_for_sample(self, after: float, timeout: float = 3.0) -> None:
        end = time.perf_counter() + timeout
        while self.proc and time.perf_counter() < end:
            if self.rows and self.rows[-1][0] > after:
                return
            time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float = None, t1: float = None):
        rows = list(self.rows)
        if t0 is not None and t1 is not None:
            before = [r for r in rows if r[0] < t0][-1:]
            during = [r for r in rows if t0 <= r[0] <= t1]
            after = [r for r in rows if r[0] > t1][:1]
            rows = before + during + after
        rows = [r for _, r in rows if len(r) > 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def max_over_ranks(ms, world, device):
    """The job's time: the slowest rank's, by an all-reduce MAX when there are several."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells, steps, world, ms_max):
    """Whole-job Gcell-updates/s: each of the `world` ranks advances its own replica of
    `cells` cells by `steps` steps within `ms_max` milliseconds."""
    return cells * steps * world / (ms_max * 1e-3) / 1e9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def device_digest():
    """Digest of the device code (the two headers every kernel is compiled from)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2206_00638_gb300", "csrc")
    for f in ("kernels.cuh", "fused.cuh"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str, depth, rows, width):
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.txt), if it
    was taken on the current device code, this workload and (one-pass kernel) this tile:
    z-block depth, rows and width."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        with open(path) as f:
            table = [l.split() for l in f if l.strip() and not l.startswith("#")]
    except OSError:
        return None
    digest = device_digest()
    for r in table:
        if (len(r) >= 7 and r[0] == kernel and r[1] == digest and r[2] == workload and r[3] in ("-", str(depth))
                and r[4] in ("-", str(rows)) and r[5] in ("-", str(width))):
            return float(r[6])
    return None


def block_workload(args):
    """The N^3 block workload named by --workload, and a description of its faces."""
    from paper_2206_00638_gb300 import workloads as wl
    if args.workload == "dielectric":
        return wl.dielectric(N=args.N, steps=args.steps), "PEC x6"
    return wl.mixed_faces(N=args.N, steps=args.steps), "PMC x, PEC y, absorbing z"


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2206_00638_gb300 import sbpsat
    from paper_2206_00638_gb300 import workloads as wl

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    w, faces = block_workload(args)
    fp16 = args.precision == "fp16"
    prec = sbpsat.FP32_FP16STORE if fp16 else sbpsat.FP32
    spec = w.blocks[0]
    cells = spec.n[0] * spec.n[1] * spec.n[2]
    stream = torch.cuda.current_stream()
    flags = sbpsat.FLAG_FDTD if args.scheme == "fdtd" else 0
    sim = sbpsat.from_workload(w, stream=stream, precision=prec, flags=flags)[0]
    nk = min(max(args.steps, 100), 400)          # steps of the per-kernel timing leg
    sim.reserve_probes(args.warmup + args.steps + nk + 8)
    if not args.no_autotune:
        sim.autotune(20)                # tile of the one-pass step: rows and depth (state unchanged)
    rows, depth, width = sim.tile()

    with ClockSampler(local) as clk:
        sim.step(args.warmup)
        torch.cuda.synchronize()
        clk.wait_for_sample(time.perf_counter())

        # headline: K whole steps, device-timed with CUDA events on the simulation's stream
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        start.record(stream)
        sim.step(args.steps)
        stop.record(stream)
        torch.cuda.synchronize()
        t_end = time.perf_counter()
        if world > 1:
            dist.barrier()
        clk.wait_for_sample(t_end)
        ms_max = max_over_ranks(start.elapsed_time(stop), world, "cuda")
        value = job_throughput(cells, args.steps, world, ms_max)
        clocks = clk.summary(t_start, t_end)

        # per-kernel durations: further steps with CUDA events around every launch
        times = sim.step_timed(nk)
    peak, peak_kind = peaks()
    nx, ny, nz = spec.n
    # Algorithmic bytes per cell-update: every field read twice (once per half-step) and
    # written once, plus the cell's eps_r: 6*3*4 + 1 = 73 B (FP32), 6*3*2 + 1 = 37 B (FP16
    # storage).  The one-pass kernel performs whole steps of its cells; the band kernels
    # the two half-steps of theirs.
    alg = 37.0 if fp16 else 73.0
    units = {   # cells each launch updates, and algorithmic bytes per cell
        "fused_interior": ((nx - 5) * (ny - 5) * (nz - 5), alg),
        # band kernels: nodes of the padded box outside the interior box of the one-pass step
        "band_h": ((nx + 2) * (ny + 2) * (nz + 2) - (nx - 6) * (ny - 6) * (nz - 6), alg / 2),
        "band_e": ((nx + 2) * (ny + 2) * (nz + 2) - (nx - 5) * (ny - 5) * (nz - 5), alg / 2),
        "h_update": (cells, alg / 2),
        "e_update": (cells, alg / 2),
    }
    moved = {"fused_interior": BYTES_FUSED, "band_h": BYTES_H, "band_e": BYTES_E, "h_update": BYTES_H,
             "e_update": BYTES_E}
    dom = max(times, key=lambda k: times[k][0] * times[k][1])
    tdom = times[dom][0]
    ucount, bpc = units[dom]
    mpc = BYTES16[dom] if fp16 else moved[dom]
    achieved = bpc * ucount / (tdom * 1e-3) / 1e9
    traffic = recorded_traffic(dom, w.name, depth, rows, width)
    launches_per_step = sum(c for _, c in times.values()) / nk
    sim.close()

    # end to end through the public API with host buffers: create (materials up),
    # initial fields up, the workload's full step count, probes and one field down
    e2e = None
    if not args.no_e2e:
        n_e2e = max(args.steps, w_default_steps(args))
        pinned = [torch.zeros(wl.field_shape(spec.n, c), dtype=torch.float32).pin_memory() for c in range(6)]
        out = torch.empty(pinned[2].shape, dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = sbpsat.Sim(spec.n, spec.h, spec.faces, eps_r=spec.eps_r, cfl=w.cfl, stream=stream, precision=prec,
                        flags=flags)
        for c in range(6):
            sbpsat._check(sbpsat.lib().sbp_set_field(s2.handle, c, pinned[c].data_ptr(), 0), "set")
        for src in spec.sources:
            s2.add_source(src.comp, src.i, src.j, src.k, src.kind, src.amp, src.tw, src.t0, src.f)
        for p in spec.probes:
            s2.add_probe(p.comp, p.i, p.j, p.k)
        s2.reserve_probes(n_e2e)
        s2.step(n_e2e)
        pr = s2.probes()
        sbpsat._check(sbpsat.lib().sbp_get_field(s2.handle, 2, out.data_ptr(), 0), "get")
        t1 = time.perf_counter()
        h2d = sum(p.numel() * 4 for p in pinned) + cells * 4
        d2h = out.numel() * 4 + pr.size * 4
        e2e = {"value": cells * n_e2e / (t1 - t0) / 1e9, "unit": "Gcell-updates/s",
               "h2d_bytes_per_step": h2d / n_e2e, "d2h_bytes_per_step": d2h / n_e2e,
               "seconds": t1 - t0, "steps": n_e2e,
               "what": "creation (material cells from pageable host memory), initial-field upload from "
                       "pinned host memory, the workload's steps, probe samples and one field back to pinned "
                       "host memory"}
        s2.close()

    serving = None
    if not args.no_serve and world == 1:
        serving = serve_stream(args)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args, budget=args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": "Gcell-updates/s", "value": value, "unit": "Gcell-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "cells": cells, "h_m": spec.h[0], "faces": faces,
                       "cfl": w.cfl, "precision": "FP32 arithmetic, FP16 storage" if fp16 else "FP32",
                       "parallelism": f"replicas x{world}", "z_block_depth": depth, "tile_rows": rows,
                       "tile_width": width,
                       "scheme": "SBP-SAT" if args.scheme == "sbp" else "FDTD (Yee) comparator",
                       "l2": "inputs_larger_than_l2 (working set %.0f MB)" % (cells * (28 if fp16 else 52) / 1e6)},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "algorithmic_bytes_per_cell": bpc,
                         "cells_per_launch": ucount, "kernel_ms": tdom,
                         "moved_bytes_per_cell": mpc,
                         "moved_frac": mpc * ucount / (tdom * 1e-3) / 1e9 / peak,
                         "traffic_over_algorithmic": (traffic / (bpc * ucount)) if traffic else None,
                         "step_frac": value / world * alg / peak,
                         "nominal_peak": HBM_NOMINAL_GBS,
                         "frac_of_nominal": achieved / HBM_NOMINAL_GBS,
                         "kernel_ms_all": {k: v[0] for k, v in times.items()}},
            "e2e": e2e,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clocks,
            "cpu_baseline": cpu,
            "serving": serving,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# the step count each block workload is stated with
STATED_STEPS = {"mixed": 1000, "dielectric": 2000}


def w_default_steps(args):
    return STATED_STEPS.get(args.workload, args.steps)


def oracle_block(w):
    import oracle
    spec = w.blocks[0]
    dt = oracle.dt_cfl(w.cfl, *spec.h)
    blk = oracle.Block(spec.n, spec.h, dt, spec.faces, eps_r=spec.eps_r)
    for s in spec.sources:
        blk.add_source(s.comp, s.i, s.j, s.k, s.kind, s.amp, s.tw, s.t0, s.f)
    return blk


def cpu_baseline(args, budget=15.0):
    """The FP64 oracle, as it stands, on the host cores: the same full-size grid as the GPU
    line, as many steps as fit in the time budget (bounded sample)."""
    import oracle

    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    w, _ = block_workload(args)
    spec = w.blocks[0]
    blk = oracle_block(w)
    cells = spec.n[0] * spec.n[1] * spec.n[2]
    t0 = time.perf_counter()
    oracle.step([blk], 1)
    t1 = time.perf_counter()
    n = max(1, min(args.steps, int(budget / max(t1 - t0, 1e-6))))
    t0 = time.perf_counter()
    oracle.step([blk], n)
    t1 = time.perf_counter()
    line = {"value": cells * n / (t1 - t0) / 1e9, "unit": "Gcell-updates/s", "cores": oracle.get_threads(),
            "kind": "oracle", "sample": f"{n} leapfrog steps of the full {w.name} grid (FP64 C oracle)",
            "seconds": t1 - t0}
    # the same oracle on one core, a shorter bounded sample (steps continue from the state above)
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.step([blk], 1)
        t1 = time.perf_counter()
        n1 = max(1, min(args.steps, int(budget / 3 / max(t1 - t0, 1e-6))))
        if n1 > 1:
            t0 = time.perf_counter()
            oracle.step([blk], n1)
            t1 = time.perf_counter()
        line["single_core"] = {"value": cells * n1 / (t1 - t0) / 1e9, "cores": 1,
                               "sample": f"{n1} leapfrog steps of the same grid", "seconds": t1 - t0}
    finally:
        oracle.set_threads(cores)
    return line


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores, on the same workload,
    metric and unit as our arm; each step is a full-grid leapfrog step, as many as fit in 150 s."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    budget = 150.0
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    w, _ = block_workload(args)
    spec = w.blocks[0]
    blk = oracle_block(w)
    cells = spec.n[0] * spec.n[1] * spec.n[2]
    tw0 = time.perf_counter()
    nw = max(1, min(args.warmup, 3))
    oracle.step([blk], nw)
    per = (time.perf_counter() - tw0) / nw
    k = max(1, min(args.steps, int(budget / max(per, 1e-6))))
    t0 = time.perf_counter()
    oracle.step([blk], k)
    t1 = time.perf_counter()
    value = cells * k / (t1 - t0) / 1e9
    line = {
        "impl": "reference", "metric": "Gcell-updates/s", "value": value, "unit": "Gcell-updates/s",
        "n_gpus": 0, "steps": k, "warmup": nw, "ms_per_step": (t1 - t0) / k * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "cells": cells, "precision": "FP64"},
        "cpu_baseline": {"value": value, "unit": "Gcell-updates/s", "cores": oracle.get_threads(),
                         "kind": "oracle",
                         "sample": f"{k} of the requested {args.steps} steps of the full {w.name} grid"},
        "e2e": {"value": value, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def serve_stream(args):
    """The serving stream run to completion three ways, end to end per request (creation and
    material upload, every step, probe samples back to the host):
    (1) plain: one grid at a time through sbp_step (the plain one-grid-per-launch FP32 path);
    (2) the continuous-batching server with every request submitted at once (closed loop);
    (3) the server with Poisson arrivals at rho times the plain throughput (p50 / p99 latency)."""
    import random

    import numpy as np
    import torch

    from paper_2206_00638_gb300 import sbpsat
    from paper_2206_00638_gb300 import workloads as wl

    reqs = wl.serving_requests(nreq=args.requests, seed=4)
    work = [int(np.prod(r["n"])) * r["steps"] for r in reqs]
    total = float(sum(work))
    stream = torch.cuda.Stream()

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in reqs:
        spec = wl.serving_spec(r)
        s = sbpsat.Sim(spec.n, spec.h, spec.faces, eps_r=spec.eps_r, cfl=0.95, stream=stream)
        for src in spec.sources:
            s.add_source(src.comp, src.i, src.j, src.k, src.kind, src.amp, src.tw, src.t0, src.f)
        for p in spec.probes:
            s.add_probe(p.comp, p.i, p.j, p.k)
        s.reserve_probes(r["steps"])
        s.step(r["steps"])
        s.probes()
        s.close()
    plain_s = time.perf_counter() - t0
    plain = total / plain_s / 1e9

    def serve(arrivals):
        srv = sbpsat.Server(stream=stream, budget_bytes=int(args.budget_gib * 2 ** 30), max_slots=args.slots,
                            chunk=32)
        tickets = []
        start = time.perf_counter()
        for q, r in enumerate(reqs):
            if arrivals is not None:
                delay = start + arrivals[q] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            tickets.append(srv.submit(wl.serving_spec(r), r["steps"]))
        srv.drain()
        res = [srv.poll(t) for t in tickets]
        cu, span = srv.stats()
        lat = np.array([x.done_s - x.submit_s for x in res]) * 1e3
        bad = sum(1 for x in res if x.status != 0)
        srv.close()
        return cu / span / 1e9, float(np.percentile(lat, 50)), float(np.percentile(lat, 99)), bad, span

    closed_v, closed_p50, closed_p99, bad1, closed_span = serve(None)
    rate = args.rho * plain * 1e9 / (total / len(reqs))      # requests per second
    rnd = random.Random(4)
    t, arr = 0.0, []
    for _ in reqs:
        t += rnd.expovariate(rate)
        arr.append(t)
    open_v, p50, p99, bad2, open_span = serve(arr)
    return {
        "workload": f"serving_stream_{len(reqs)}req", "unit": "Gcell-updates/s",
        "cells_per_axis": "U{32..192}", "steps": "U{500..4000}", "faces": "PEC or absorbing, p = 1/2 each",
        "slots": args.slots, "hbm_budget_gib": args.budget_gib, "chunk_steps": 32,
        "total_cell_updates": total,
        "plain_one_grid_per_launch": plain, "plain_seconds": plain_s,
        "batched_closed_loop": closed_v, "batched_over_plain": closed_v / plain, "closed_seconds": closed_span,
        "closed_p50_ms": closed_p50, "closed_p99_ms": closed_p99,
        "poisson": {"rho": args.rho, "requests_per_s": rate, "aggregate": open_v, "p50_ms": p50, "p99_ms": p99,
                    "seconds": open_span},
        "failed_requests": bad1 + bad2,
        "latency": "arrival (submit) to result on the host, end to end",
    }


def run_blocks(args):
    """Throughput of the other block workloads, device-timed like the default line: the two
    192x192x96 blocks joined on z by the interface SAT (FP32, stepped as a group) and the PEC
    cavity (20x16x12, FP64, the in-place path)."""
    import torch

    from paper_2206_00638_gb300 import sbpsat
    from paper_2206_00638_gb300 import workloads as wl

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if args.workload == "twoblock":
        w, prec = wl.two_block(steps=args.steps), sbpsat.FP32
    else:
        w, prec = wl.cavity(steps=args.steps), sbpsat.FP64
    stream = torch.cuda.current_stream()
    sims = sbpsat.from_workload(w, stream=stream, precision=prec)
    for s in sims:
        s.reserve_probes(args.warmup + args.steps + 8)
        if prec != sbpsat.FP64 and not args.no_autotune:
            s.autotune(5)
    sbpsat.step_group(sims, args.warmup)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        clk.wait_for_sample(time.perf_counter())
        t0 = time.perf_counter()
        start.record(stream)
        sbpsat.step_group(sims, args.steps)
        stop.record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        clk.wait_for_sample(t1)
        clocks = clk.summary(t0, t1)
    ms = start.elapsed_time(stop)
    cells = w.cells()
    for s in sims:
        s.close()
    line = {
        "metric": "Gcell-updates/s", "value": cells * args.steps / (ms * 1e-3) / 1e9, "unit": "Gcell-updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == sbpsat.FP64 else "f32", "data": "synthetic",
        "config": {"workload": w.name, "cells": cells, "blocks": len(sims),
                   "precision": "FP64" if prec == sbpsat.FP64 else "FP32"},
        "clocks": clocks,
    }
    print(json.dumps(line))


def run_serve(args):
    """The serving stream alone, as its own JSON line."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    s = serve_stream(args)
    line = {
        "metric": "Gcell-updates/s (serving, aggregate, end to end)", "value": s["batched_closed_loop"],
        "unit": "Gcell-updates/s", "n_gpus": 1, "steps": args.requests, "warmup": 0, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": s["workload"]}, "serving": s,
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload in ("twoblock", "cavity"):
        run_blocks(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
