#!/usr/bin/env python
"""Benchmark of the screen-space sampler optimiser on GB300.

Workload (one step): optimise a batch of 128 x 128 tiles, each a rank-1 lattice of N = 64 points
per pixel scored against T = 1024 random Heavisides (int8 counts), Eq. 1 weight sigma 2.1 with
radius 6, for 2000 passes of the parallel swap optimiser; the step re-initialises every tile
from a new seed (shifts, integrands, permutation, counts), runs the passes, evaluates Eq. 1 and
gathers the optimised shifts.  Inputs are synthetic by construction (random Heavisides, Philox
shifts), so no dataset is involved.

Metric: move proposals evaluated per second (valid couples whose swap energy was evaluated),
whole job over all ranks; optimised tiles per second is reported beside it.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W_TILE = H_TILE = 128
N_POINTS, T_INTEGRANDS, SIGMA, RADIUS, SWEEPS = 64, 1024, 2.1, 6, 2000
WORKLOAD = ("128x128 toroidal tile, rank-1 lattice N=64 (Korobov g=19), T=1024 random "
            "Heavisides (int8 counts), Eq.1 weight exp(-d^2/2.1^2) radius 6, 2000 passes")
METRIC = "move proposals evaluated/sec"
UNIT = "proposals/s"
STENCIL_OFFSETS = 112           # neighbours within radius 6 on a tile >= 13 x 13
L2_FLUSH_BYTES = 256 << 20      # > 129 MB L2
# nominal int8 dot-product (IDP4A) peak: 152 SMs x 64 IDP4A/clk x 4 MAC x 2.07 GHz
DP4A_PEAK_TOPS = 152 * 64 * 4 * 2.07e9 / 1e12
# 16-bit counts: one multiply-accumulate per IMAD, 64 IMAD/clk/SM
IMAD_PEAK_TOPS = 152 * 64 * 2.07e9 / 1e12
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
# DRAM bytes (read + write) per tile-pass of the persistent sweep kernel, 8x8 CTA shape, int8
# counts, working set larger than L2: one ncu capture of 16 tiles x 6 passes (the profile summary
# of k_persistent for 128x128 N=64 T=1024); a launch's traffic scales with its tile-passes
TRAFFIC_PER_TILE_PASS = (1683.924e6 + 58.356e6) / (16 * 6)
PASSES_PER_LAUNCH = 500
# DRAM bytes (read + write) per tile-pass of the tensor-core stencil on the same tiles: one ncu
# capture of one launch over 16 tiles (the profile summary of k_tc_stencil for 128x128 N=64
# T=1024); a launch's traffic scales with the tiles it covers
TC_TRAFFIC_PER_TILE_PASS = (349.900032e6 + 5.298176e6) / 16
# shared-memory wavefront rate: 128 B per SM clock, measured 120 B/clk/SM by a probe
SMEM_PEAK_TBS = 152 * 120 * 2.07e9 / 1e12


# ------------------------------------------------------------------------------------------------
# host-side helpers (no GPU needed; covered by CPU tests)
# ------------------------------------------------------------------------------------------------
def tile_seed(rank: int, step: int, tile: int, tiles_per_rank: int) -> int:
    """Seed of one tile: every rank, step and tile gets its own problem (weak scaling)."""
    return 1_000_003 * rank + tiles_per_rank * step + tile + 1


def proposals_per_tile(sweeps: int = SWEEPS) -> int:
    P = W_TILE * H_TILE
    return sweeps * P // 8  # P is a power of two: every couple of every pass is valid


def all_reduce_list(values, dist, device: str, op: str = "max") -> list[float]:
    """Reduce a few host numbers over all ranks (max for times: the slowest rank bounds the job;
    sum for work done)."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()]


def merge_serving(summary: dict, dist, device: str) -> dict:
    """Whole-job serving figures: latency percentiles of every rank's requests pooled (the
    per-request latencies are all-gathered), the slowest rank's makespan, summed work and
    request counts.  The raw per-request lists are dropped from the result."""
    from paper_2105_12620_gb300 import serving as srv
    out = {k: v for k, v in summary.items() if k not in ("latencies_s", "queue_s")}
    lat, wait = list(summary.get("latencies_s", [])), list(summary.get("queue_s", []))
    if dist is not None:
        gathered = [None] * dist.get_world_size()
        dist.all_gather_object(gathered, (lat, wait))
        lat = [v for g in gathered for v in g[0]]
        wait = [v for g in gathered for v in g[1]]
        (out["makespan_s"],) = all_reduce_list([summary["makespan_s"]], dist, device, "max")
        props, done, reqs = all_reduce_list(
            [summary["proposals_per_s"] * summary["makespan_s"], summary["completed"],
             summary["requests"]], dist, device, "sum")
        out["proposals_per_s"] = props / out["makespan_s"]
        out["served_req_per_s"] = done / out["makespan_s"]
        out["completed"], out["requests"] = int(done), int(reqs)
    out.update(srv.latency_percentiles(lat, wait))
    out["latency_samples"] = len(lat)
    return out


def parse_clocks(text: str, gpu_index: int | None = None) -> dict:
    rows = []
    for line in text.strip().splitlines():
        if not line or line.startswith("index"):
            continue
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            idx = int(f[0])
            sm = float(f[1].split()[0])
            smax = float(f[2].split()[0])
        except ValueError:
            continue
        if gpu_index is not None and idx != gpu_index:
            continue
        rows.append((sm, smax, f[5:9]))
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    reasons = sorted({REASONS[i] for _, _, r in rows for i in range(4) if r[i] == "Active"})
    return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
            "reasons": reasons, "samples": len(rows)}


class ClockSampler:
    """nvidia-smi sampling every 200 ms during the timed region."""

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="bn_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={SMI_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200",
                                          "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self, gpu_index: int | None) -> dict:
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        text = open(self.path).read() if self.path and os.path.exists(self.path) else ""
        if self.path and os.path.exists(self.path):
            os.unlink(self.path)
        return parse_clocks(text, gpu_index)


def physical_gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if local_rank < len(ids) and ids[local_rank].strip().isdigit():
        return int(ids[local_rank])
    return local_rank


# ------------------------------------------------------------------------------------------------
# reference arm and CPU baseline: the FP64 oracle on the host cores
# ------------------------------------------------------------------------------------------------
def oracle_rate(n_sweeps: int, seed: int = 1) -> tuple[float, float, str]:
    """Proposals/s of the plain C oracle on one tile of the workload (single thread)."""
    import oracle
    tile = oracle.OracleTile(W_TILE, H_TILE, N_POINTS, T_INTEGRANDS, seed=seed, sigma=SIGMA,
                             radius=RADIUS)
    t0 = time.perf_counter()
    props = 0
    for _ in range(n_sweeps):
        lg = tile.sweep()
        props += int((lg.flags & 1).sum())
    dt = time.perf_counter() - t0
    sample = f"one 128x128 tile (N=64, T=1024) after initialisation, {n_sweeps} passes"
    return props / dt, dt, sample


def _oracle_tile_passes(seed: int, n_sweeps: int) -> tuple[int, float]:
    """(valid proposals, seconds) of n_sweeps oracle passes on one tile (one process)."""
    import oracle
    tile = oracle.OracleTile(W_TILE, H_TILE, N_POINTS, T_INTEGRANDS, seed=seed, sigma=SIGMA,
                             radius=RADIUS)
    t0 = time.perf_counter()
    props = 0
    for _ in range(n_sweeps):
        props += int((tile.sweep().flags & 1).sum())
    return props, time.perf_counter() - t0


def oracle_rate_all_cores(n_sweeps: int) -> tuple[float, int, float, str]:
    """Proposals/s of the oracle with one independent tile per host core (spawned processes,
    each single-threaded; only the passes are timed)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_tile_passes, [(100 + i, n_sweeps) for i in range(cores)])
    props = sum(r[0] for r in res)
    span = max(r[1] for r in res)
    sample = (f"{cores} independent 128x128 tiles (N=64, T=1024), one per core, {n_sweeps} passes "
              "each after initialisation")
    return props / span, cores, span, sample


def run_reference(args) -> int:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    per_step = 3  # passes per step: a bounded sample of the workload (~2 s of CPU each)
    import oracle
    tile = oracle.OracleTile(W_TILE, H_TILE, N_POINTS, T_INTEGRANDS, seed=1, sigma=SIGMA,
                             radius=RADIUS)
    for _ in range(args.warmup):
        tile.sweep()
    times, props = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            props += int((tile.sweep().flags & 1).sum())
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = props / total
    sample = f"{per_step} passes of one 128x128 tile (N=64, T=1024) per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference": "plain C FP64 oracle, single thread",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def plain_per_tile(pkg, stream, rank, sweeps: int = 512, reps: int = 3) -> dict:
    """The plain schedule (three launches per pass, one warp per couple) on one tile, replayed
    from CUDA graphs of 32 passes, and with every kernel launched directly."""
    import torch
    t = pkg.Sampler(W_TILE, H_TILE, N_POINTS, T_INTEGRANDS, seed=tile_seed(rank, 99, 0, 1),
                    sigma=SIGMA, radius=RADIUS, schedule=pkg.BN_SCHEDULE_PLAIN, stream=stream)
    rates = {}
    with torch.cuda.stream(stream):
        for graph in (32, 0):
            t.set_graph_passes(graph)
            t.optimize(96, stats=False)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                t.optimize(sweeps, stats=False)
            b.record(stream)
            torch.cuda.synchronize()
            rates[graph] = reps * proposals_per_tile(sweeps) / (a.elapsed_time(b) / 1000.0)
    t.close()
    return {"value": rates[32], "unit": UNIT, "tiles_per_s": rates[32] / proposals_per_tile(),
            "direct_launches": rates[0],
            "note": f"1 tile, plain schedule, {reps}x{sweeps} passes (no re-initialisation); "
                    "value: CUDA graphs of 32 passes, direct_launches: one launch per kernel"}


def spectrum_summary(pkg, stream) -> dict:
    """Fig. 1b on one tile of the workload: the error power of the lowest frequency rings
    (radius 1 .. side / 8 cycles per tile) before and after the optimisation's pass budget."""
    import numpy as np
    with pkg.Sampler(W_TILE, H_TILE, N_POINTS, T_INTEGRANDS, seed=1, sigma=SIGMA, radius=RADIUS,
                     stream=stream) as s:
        p0, c = s.spectrum("heaviside")
        s.optimize(SWEEPS, stats=False)
        p1, _ = s.spectrum("heaviside")
    low = slice(1, W_TILE // 8 + 1)
    lo0, lo1 = float((p0[low] * c[low]).sum()), float((p1[low] * c[low]).sum())
    return {"low_rings": [1, W_TILE // 8], "initial": lo0, "optimised": lo1,
            "ratio": lo1 / lo0 if lo0 > 0 else None,
            "total_initial": float((p0 * c).sum()), "total_optimised": float((p1 * c).sum()),
            "config": f"one {W_TILE}x{H_TILE} tile, N={N_POINTS}, T={T_INTEGRANDS} Heavisides, "
                      f"{SWEEPS} passes; power |DFT|^2 / (W H) of the error tiles, mean over "
                      "integrands, summed over the rings"}


def run_serving(pkg, args, rank: int, local: int, world: int, dist, n_requests: int | None = None,
                rate: float | None = None) -> dict:
    """Bounded run of the serving loop: a Poisson stream of mixed requests per GPU (weak
    scaling: every rank serves its own stream); latency percentiles pool every rank's
    requests."""
    from paper_2105_12620_gb300 import serving as srv

    n_requests = args.serving_requests if n_requests is None else n_requests
    rate = args.serving_rate if rate is None else rate
    reqs = srv.draw_requests(n_requests, rate, seed=1000 + rank)
    with pkg.Server(max_slots=args.serving_slots, sweeps_per_chunk=args.serving_chunk,
                    device=local) as sv:
        summary = srv.run_load(sv, reqs, timeout_s=args.serving_timeout)
        summary["server"] = sv.stats()
    summary = merge_serving(summary, dist, "cuda")
    summary["config"] = {
        "stream": f"Poisson {rate:g} req/s per GPU, {n_requests} "
                  "requests (bounded run), side log-uniform 32..512, N in {16,64,256}, T=1024, "
                  "1 or 2 pairs, pass budget uniform 500..5000",
        "max_slots": args.serving_slots, "sweeps_per_chunk": args.serving_chunk,
        "memory_budget": "80% of free device memory", "latency": "submit to done",
        "schedule": "tensor-core batch for the request signatures the autotuner assigns to it "
                    "(timed once per signature), the other requests fused in a second batch"}
    return summary


def workload_tiles(args):
    """(tiles, description) of the benchmarked workload; sweeps override the pass budget."""
    from paper_2105_12620_gb300 import workloads as wl
    if args.workload == "c2":
        tiles = wl.c2(args.tiles)
        desc = WORKLOAD
    elif args.workload == "c3":
        tiles = wl.c3()
        desc = ("256x256 toroidal tile, two pairs of dimensions, rank-1 lattice N=256 (g=71), "
                "T=512 Heavisides per pair (int16 counts), Eq.1 sigma 2.1 radius 6, 4000 passes")
    else:
        tiles = wl.c4()
        desc = ("96 tiles, side in {32,64,128,256}, N in {4,16,64}, T in {256,1024} (Philox "
                "seed 0), Eq.1 sigma 2.1 radius 6, 2000 passes, fused in one batch")
    if args.sweeps:
        desc = desc.replace(f"{tiles[0].sweeps} passes", f"{args.sweeps} passes")
        tiles = [wl.Tile(t.width, t.height, t.n_points, t.n_integrands, t.n_pairs, args.sweeps)
                 for t in tiles]
    return tiles, desc


SCHEDULE_NAMES = {1: "plain", 2: "persistent", 3: "tensor"}


def schedule_desc(chosen: dict) -> dict:
    """The chosen schedule for the JSON line (CTA shape and chunk split: persistent only)."""
    kind = SCHEDULE_NAMES.get(chosen["kind"], "?")
    out = {"kind": kind}
    if kind == "persistent":
        out.update({"block": list(chosen["shape"][:2]), "threads": chosen["shape"][2],
                    "tsplit": chosen["tsplit"]})
    if kind == "tensor":
        out["product"] = "tcgen05.mma kind::f16, M = 128 patch pixels, N <= 160, K = 16"
    out["chosen_by"] = chosen.get("chosen_by", "autotuner")
    return out


def measured_peak(key: str):
    """(value, provenance) of a peak from the measured file, else the recipe fallback."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)[key]), "of measured"
    except (OSError, KeyError, ValueError):
        return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "hbm_gbs": 6800.0}[key], "of fallback"


def kernel_roofline(ktimes: dict, specs, split_steps: int, sweeps: int, args, chosen, pkg):
    """Roofline of the dominant kernel of the kernel-split run.

    Algorithmic work of a proposal: 2 sides x 112 neighbours x T multiply-accumulates (the
    swap terms of Eq. 1).  Algorithmic bytes of a tile-pass: the P x T count bytes every pass
    must read (every pixel neighbours some proposed pixel).  Both over the kernel's average
    launch duration (CUDA events on its stream)."""
    if not ktimes:
        return None
    name, (nl, tms) = max(ktimes.items(), key=lambda kv: kv[1][1])
    total_ops = split_steps * sum(t.proposals() * 2 * STENCIL_OFFSETS * t.n_integrands
                                  for t in specs)
    count_bytes = split_steps * sweeps * sum(
        t.width * t.height * t.n_integrands * (2 if t.n_points > 64 else 1) * t.n_pairs
        for t in specs)
    wide = any(t.n_points > 64 for t in specs)
    secs = tms / 1000.0
    hbm_peak, hbm_src = measured_peak("hbm_gbs")
    all_ms = sum(v[1] for v in ktimes.values())
    hbm = {"achieved": count_bytes / secs / 1e9, "peak": hbm_peak, "unit": "GB/s",
           "frac": count_bytes / secs / 1e9 / hbm_peak,
           "pass_frac": count_bytes / (all_ms / 1000.0) / 1e9 / hbm_peak,
           "note": "algorithmic bytes: the P x T count bytes a pass reads, over this kernel's "
                   "time (frac) and over every kernel of the pass (pass_frac); peak = HBM copy "
                   + hbm_src}
    if name == "stencil_tensor":
        # f16 products on the tensor pipe: useful FLOPs (2 per multiply-accumulate the stencil
        # keeps; the products outside the radius are not counted) against the measured dense
        # bf16 peak sustained over seconds (the kernel runs inside a seconds-long step; f16
        # runs at the bf16 rate)
        tpeak, tsrc = measured_peak("bf16_tflops_sustained")
        tf = 2.0 * total_ops / secs / 1e12
        alu_peak = IMAD_PEAK_TOPS if wide else DP4A_PEAK_TOPS
        traffic = None
        if args.workload == "c2" and not wide:
            # per launch: the tile-passes of the split run over its stencil launches
            traffic = TC_TRAFFIC_PER_TILE_PASS * len(specs) * split_steps * sweeps / nl
        return {"kernel": name, "bound": "tensor", "achieved": tf, "peak": tpeak,
                "unit": "TFLOP/s", "frac": tf / tpeak, "traffic": traffic,
                "note": "useful f16 FLOPs of the stencil (2 per kept product); peak = dense "
                        "bf16 sustained " + tsrc,
                "launches": nl, "avg_launch_ms": tms / nl, "share": tms / max(all_ms, 1e-9),
                "hbm": hbm,
                "int8_equivalent": {"achieved": total_ops / secs / 1e12, "peak": alu_peak,
                                    "unit": "TOP/s",
                                    "frac": total_ops / secs / 1e12 / alu_peak}}
    peak = IMAD_PEAK_TOPS if wide else DP4A_PEAK_TOPS
    achieved = total_ops / secs / 1e12
    traffic = None
    sched = chosen or {}
    if (args.workload == "c2" and not wide and sched.get("kind") == pkg.BN_SCHEDULE_PERSISTENT
            and tuple(sched.get("shape", ())[:2]) == (8, 8)):
        traffic = TRAFFIC_PER_TILE_PASS * len(specs) * min(sweeps, PASSES_PER_LAUNCH)
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TOP/s", "frac": achieved / peak, "traffic": traffic,
            "note": ("op = one int16 multiply-accumulate; peak = IMAD nominal "
                     "(152 SMs x 64/clk x 2.07 GHz)") if wide else
                    ("op = one int8 multiply-accumulate; peak = IDP4A nominal "
                     "(152 SMs x 64/clk x 4 x 2.07 GHz)"),
            "launches": nl, "avg_launch_ms": tms / nl, "share": tms / max(all_ms, 1e-9),
            "hbm": hbm}


def run_extra_workload(pkg, args, name: str, stream, rank: int, world: int, dist) -> dict:
    """One more workload timed like the headline (autotuned schedule, CUDA-graph sweeps, L2
    flushed between steps, device events around each step), reported beside it: the 256 x 256
    two-pair tile with int16 counts (c3) or the 96 mixed tiles (c4)."""
    import torch

    sub = argparse.Namespace(**vars(args))
    sub.workload, sub.sweeps = name, 0
    specs, desc = workload_tiles(sub)
    B = len(specs)
    sweeps = specs[0].sweeps
    tiles = [pkg.Sampler(t.width, t.height, t.n_points, t.n_integrands,
                         seed=tile_seed(rank, 0, i, B), n_pairs=t.n_pairs, sigma=SIGMA,
                         radius=RADIUS, stream=stream)
             for i, t in enumerate(specs)]
    batch = pkg.Batch(tiles, stream=stream) if B > 1 else None
    chosen = batch.autotune(20) if batch is not None else tiles[0].autotune(20)
    energy_dev = torch.empty(sum(t.n_pairs for t in specs), dtype=torch.float64, device="cuda")
    energy_off = [0]
    for t in specs:
        energy_off.append(energy_off[-1] + t.n_pairs)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(k: int):
        for i, t in enumerate(tiles):
            t.reset(tile_seed(rank, k, i, B))
        (batch if batch is not None else tiles[0]).optimize(sweeps, stats=False)
        for i, t in enumerate(tiles):
            t.energy_into(energy_dev[energy_off[i]:energy_off[i + 1]].data_ptr())

    steps = args.extra_steps
    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            flush.zero_()
            step(k)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            step(args.warmup + k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    (total_ms,) = all_reduce_list([sum(a.elapsed_time(b) for a, b in ev)], dist, "cuda", "max")
    if batch is not None:
        batch.close()
    for t in tiles:
        t.close()
    props = sum(t.proposals() for t in specs)
    return {"value": world * props * steps / (total_ms / 1000.0), "unit": UNIT,
            "tiles_per_s": world * B * steps / (total_ms / 1000.0),
            "ms_per_step": total_ms / steps, "steps": steps, "warmup": args.warmup,
            "dtype": "int16" if any(t.n_points > 64 for t in specs) else "int8",
            "config": {"workload": desc, "tiles_per_gpu": B, "sweeps": sweeps,
                       "schedule": schedule_desc(chosen),
                       "timing": "device events around each step; sweeps replayed from CUDA "
                                 "graphs; L2 flushed between steps (256 MB write)"}}


def run_ours(args) -> int:
    import torch

    import paper_2105_12620_gb300 as pkg
    from paper_2105_12620_gb300 import build as pkg_build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus != world and world > 1:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE {world}")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not pkg_build.up_to_date():
        pkg_build.build()
    if dist is not None:
        dist.barrier()
    pkg.load()
    from paper_2105_12620_gb300 import _lib as L

    stream = torch.cuda.Stream()
    specs, desc = workload_tiles(args)
    B = len(specs)
    sweeps = specs[0].sweeps  # every tile of a workload has the same pass budget
    schedule = {"auto": pkg.BN_SCHEDULE_AUTO, "plain": pkg.BN_SCHEDULE_PLAIN,
                "persistent": pkg.BN_SCHEDULE_PERSISTENT,
                "tensor": pkg.BN_SCHEDULE_TENSOR}[args.schedule]
    tiles = [pkg.Sampler(t.width, t.height, t.n_points, t.n_integrands,
                         seed=tile_seed(rank, 0, i, B), n_pairs=t.n_pairs, sigma=SIGMA,
                         radius=RADIUS, schedule=schedule, stream=stream)
             for i, t in enumerate(specs)]
    batch = pkg.Batch(tiles, stream=stream) if B > 1 else None
    chosen = None
    if args.block:
        bx, by = (int(v) for v in args.block.split("x"))
        for obj in ([batch] if batch is not None else tiles):
            obj.set_schedule(pkg.BN_SCHEDULE_PERSISTENT, (bx, by, args.threads, args.spw),
                             args.tsplit)
        chosen = (batch if batch is not None else tiles[0]).get_schedule()
        chosen["chosen_by"] = "command line"
    elif args.schedule == "auto":
        # untimed: trial passes on a scratch copy pick the CTA shape / chunk split
        chosen = batch.autotune(20) if batch is not None else tiles[0].autotune(20)
    shift_floats = [t.width * t.height * 2 * t.n_pairs for t in specs]
    shifts_dev = torch.empty(sum(shift_floats), dtype=torch.float32, device="cuda")
    shift_off = [0]
    for n in shift_floats:
        shift_off.append(shift_off[-1] + n)
    energy_dev = torch.empty(sum(t.n_pairs for t in specs), dtype=torch.float64, device="cuda")
    energy_off = [0]
    for t in specs:
        energy_off.append(energy_off[-1] + t.n_pairs)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def optimize_all():
        if batch is not None:
            batch.optimize(sweeps, stats=False)
        else:
            tiles[0].optimize(sweeps, stats=False)

    def step(k: int):
        for i, t in enumerate(tiles):
            t.reset(tile_seed(rank, k, i, B))
        optimize_all()
        for i, t in enumerate(tiles):
            t.energy_into(energy_dev[energy_off[i]:energy_off[i + 1]].data_ptr())
            t.shifts_into(shifts_dev[shift_off[i]:].data_ptr(), shift_floats[i])

    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            flush.zero_()
            step(k)
        stream.synchronize()
        # timed region: the library as a user runs it (sweeps replayed from CUDA graphs, no
        # per-kernel events)
        launches0 = L.load().bn_launch_counter()
        clocks = ClockSampler()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step(args.warmup + k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        clock_info = clocks.stop(physical_gpu_index(local))
        launches = L.load().bn_launch_counter() - launches0
        step_ms = [a.elapsed_time(b) for a, b in ev]
        local_ms = sum(step_ms)
        # kernel split: the same steps once more with every kernel of a pass bracketed by CUDA
        # events on the launching stream (direct launches: events cannot sit between the
        # kernels of a replayed graph); the dominant kernel's duration for the roofline
        split_steps = min(args.steps, args.split_steps)
        tiles[0].set_kernel_timing(2)
        tiles[0].kernel_times()
        split_ms = 0.0
        for k in range(split_steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(args.warmup + args.steps + k)
            b.record(stream)
            b.synchronize()
            split_ms += a.elapsed_time(b)
        ktimes = tiles[0].kernel_times()
        tiles[0].set_kernel_timing(False)
        # end to end through the public API with host buffers (pinned staging inside)
        e2e_ms = []
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i, t in enumerate(tiles):
                t.reset(tile_seed(rank, 10_000 + k, i, B))
            optimize_all()
            host_shifts = [t.shifts() for t in tiles]
            host_energy = [t.energy() for t in tiles]
            e2e_ms.append(1000 * (time.perf_counter() - t0))
        del host_energy, host_shifts
    total_ms, e2e_total = all_reduce_list([local_ms, sum(e2e_ms)], dist, "cuda", "max")
    props_step = sum(t.proposals() for t in specs)
    value = world * props_step * args.steps / (total_ms / 1000.0)
    e2e_value = world * props_step * args.steps / (e2e_total / 1000.0)
    roofline = kernel_roofline(ktimes, specs, split_steps, sweeps, args, chosen, pkg)

    plain = None
    if not args.no_plain and rank == 0 and args.workload == "c2":
        plain = plain_per_tile(pkg, stream, rank)
    spectrum = None
    if rank == 0 and args.workload == "c2" and not args.no_plain:
        spectrum = spectrum_summary(pkg, stream)
    extra = {}
    if args.workload == "c2":
        for name in args.extra_workloads.split(","):
            if name and name != "none":
                extra[name] = run_extra_workload(pkg, args, name, stream, rank, world, dist)
    serving = serving_light = None
    if args.serving_requests > 0 and args.workload == "c2":
        serving = run_serving(pkg, args, rank, local, world, dist)
        if args.serving_light_requests > 0:
            # a stream the GPU keeps up with: latencies are service times, not queueing
            serving_light = run_serving(pkg, args, rank, local, world, dist,
                                        args.serving_light_requests, args.serving_light_rate)
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            rate_all, cores, secs_all, sample_all = oracle_rate_all_cores(args.cpu_sweeps)
            rate, secs, sample = oracle_rate(args.cpu_sweeps)
            cpu = {"value": rate_all, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": sample_all, "seconds": secs_all,
                   "single_thread": {"value": rate, "cores": 1, "sample": sample,
                                     "seconds": secs}}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int16" if any(t.n_points > 64 for t in specs) else "int8",
            "data": "synthetic",
            "config": {"workload": desc, "tiles_per_gpu": B, "sweeps": sweeps,
                       "schedule": args.schedule if chosen is None else
                       schedule_desc(chosen),
                       "objective": "raise Eq. 1 (blue-noise direction; the printed 'reduce' "
                                    "is BN_OBJECTIVE_LITERAL)",
                       "commit": "non-interacting improving couples",
                       "timing": "device events around each step; sweeps replayed from CUDA "
                                 "graphs; kernel split from %d further steps with every kernel "
                                 "bracketed by events" % split_steps,
                       "parallelism": f"independent tiles x{world}",
                       "l2": "flushed between steps (256 MB write)"},
            "tiles_per_s": world * B * args.steps / (total_ms / 1000.0),
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": sum(int(t.info.reset_h2d_bytes) for t in tiles),
                    "d2h_bytes_per_step": sum(4 * n for n in shift_floats) + 8 * energy_off[-1]},
            "gpu_launches": int(launches),
            "clocks": {k: clock_info[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "roofline": roofline,
            "kernel_ms": {k: {"launches": v[0], "total_ms": v[1]} for k, v in ktimes.items()},
            "kernel_split_ms_per_step": split_ms / max(split_steps, 1),
            "cpu_baseline": cpu,
            "plain_per_tile": plain,
            "spectrum": spectrum,
            "serving": serving,
            "serving_light": serving_light,
        }
        for name, res in extra.items():
            line["workload_" + name] = res
        print(json.dumps(line), flush=True)
    if batch is not None:
        batch.close()
    for t in tiles:
        t.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def report_kernels(args) -> int:
    """One timing of each kernel outside the sweep, on one 512 x 512 tile (N = 64, T = 1024,
    256 MiB of counts): re-initialisation (dominated by the counts), Eq. 1, the criterion on
    Heavisides and on bumps, and the renderer lookup for a 1920 x 1080 screen."""
    import torch

    import paper_2105_12620_gb300 as pkg
    from paper_2105_12620_gb300 import build as pkg_build
    pkg_build.build()
    pkg.load()
    W = H = 512
    P = W * H
    stream = torch.cuda.Stream()
    s = pkg.Sampler(W, H, N_POINTS, T_INTEGRANDS, seed=1, sigma=SIGMA, radius=RADIUS,
                    stream=stream)
    energy = torch.empty(1, dtype=torch.float64, device="cuda")
    SW, SH, NS = 1920, 1080, 16
    samples = torch.empty(SW * SH * NS * 2, dtype=torch.float32, device="cuda")

    def device_ms(fn, reps=3):
        fn()
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    def host_ms(fn, reps=2):
        fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        return 1000 * (time.perf_counter() - t0) / reps

    with torch.cuda.stream(stream):
        t_init = device_ms(lambda: s.reset(1))
        t_energy = device_ms(lambda: s.energy_into(energy.data_ptr()))
        t_samples = device_ms(lambda: s.samples_into(samples.data_ptr(), samples.numel(), 0, 0,
                                                     SW, SH, 0, NS, 2))
    t_crit = host_ms(lambda: s.criterion([1.0, 4.0], "heaviside", 128))
    t_bump = host_ms(lambda: s.criterion([1.0], "gaussian", 32))
    s.close()
    out = {
        "report": "kernels outside the sweep", "tile": "512x512, N=64, T=1024 (256 MiB of int8 counts)",
        "reinit": {"ms": t_init, "threshold_tests_per_s": P * N_POINTS * T_INTEGRANDS / t_init * 1e3,
                   "note": "shifts, Heavisides, permutation, state, counts (P*N*T tests)"},
        "energy": {"ms": t_energy,
                   "bytes_per_s": P * STENCIL_OFFSETS * T_INTEGRANDS / t_energy * 1e3,
                   "note": "one byte of a neighbour's counts per (pixel, offset, integrand), from L2"},
        "criterion_heaviside": {"ms": t_crit, "integrands": 128, "sigmas": [1.0, 4.0],
                                "note": "FP64, host call incl. scratch allocation"},
        "criterion_bumps": {"ms": t_bump, "integrands": 32, "sigmas": [1.0],
                            "note": "FP64, N exp per pixel and bump"},
        "samples": {"ms": t_samples, "bytes_per_s": samples.numel() * 4 / t_samples * 1e3,
                    "screen": f"{SW}x{SH}, {NS} samples, 2 dimensions"},
    }
    print(json.dumps(out), flush=True)
    return 0


def report_modes(args) -> int:
    """Eq. 1 and the filtered error along the passes for the two commit rules on one 128 x 128
    tile: keep only non-interacting improving couples, or every improving couple (the paper's
    GPU optimiser, which may move Eq. 1 the wrong way at first)."""
    import paper_2105_12620_gb300 as pkg
    from paper_2105_12620_gb300 import build as pkg_build
    pkg_build.build()
    pkg.load()
    every, total = 100, args.sweeps or SWEEPS
    out = {"report": "commit rule", "workload": WORKLOAD.rsplit(",", 1)[0],
           "every": every, "passes": total, "sigmas": [1.0, 2.0, 4.0, 8.0]}
    for name, mode in (("noninteracting", pkg.BN_MODE_NONINTERACTING),
                       ("concurrent", pkg.BN_MODE_CONCURRENT)):
        s = pkg.Sampler(W_TILE, H_TILE, N_POINTS, T_INTEGRANDS, seed=1, sigma=SIGMA,
                        radius=RADIUS, mode=mode)
        trace, worse = [float(s.energy()[0])], 0
        committed = 0
        for _ in range(total // every):
            st = s.optimize(every)
            committed += st.committed
            trace.append(float(s.energy()[0]))
        # passes whose own commits lowered Eq. 1 (objective: raise it)
        s2 = pkg.Sampler(W_TILE, H_TILE, N_POINTS, T_INTEGRANDS, seed=1, sigma=SIGMA,
                         radius=RADIUS, mode=mode)
        prev = float(s2.energy()[0])
        for _ in range(200):
            s2.optimize(1, stats=False)
            e = float(s2.energy()[0])
            worse += e < prev
            prev = e
        s2.close()
        out[name] = {"energy": trace, "committed": int(committed),
                     "passes_that_lowered_eq1_of_first_200": int(worse),
                     "rmse_initial_vs_final": None}
        crit = s.criterion(out["sigmas"])
        s.reset(1)
        out[name]["rmse_initial_vs_final"] = [list(map(float, s.criterion(out["sigmas"]))),
                                              list(map(float, crit))]
        s.close()
    print(json.dumps(out), flush=True)
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tiles", type=int, default=64, help="128x128 tiles per GPU per step")
    ap.add_argument("--workload", choices=["c2", "c3", "c4"], default="c2",
                    help="c2: 128x128 N=64 T=1024 tiles (default); c3: 256x256 N=256, two "
                         "pairs x T=512; c4: 96 mixed tiles")
    ap.add_argument("--sweeps", type=int, default=0, help="pass budget (0: the workload's)")
    ap.add_argument("--report", choices=["modes", "kernels"], default=None,
                    help="modes: Eq. 1 along the passes for both commit rules (no timing); "
                         "kernels: one timing of each kernel outside the sweep")
    ap.add_argument("--schedule", choices=["auto", "plain", "persistent", "tensor"],
                    default="auto")
    ap.add_argument("--cpu-sweeps", type=int, default=20)
    ap.add_argument("--split-steps", type=int, default=2,
                    help="steps of the kernel-split run (every kernel timed by events)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--block", default="", help="force a persistent CTA block, e.g. 8x8")
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--spw", type=int, default=4)
    ap.add_argument("--tsplit", type=int, default=1)
    ap.add_argument("--extra-workloads", default="c3,c4",
                    help="workloads timed after the headline and reported beside it (c3, c4; "
                         "'none' skips them)")
    ap.add_argument("--extra-steps", type=int, default=2,
                    help="timed steps of each extra workload (warm-up: --warmup)")
    ap.add_argument("--serving-requests", type=int, default=500,
                    help="requests of the bounded serving run (0 skips it)")
    ap.add_argument("--serving-rate", type=float, default=200.0, help="Poisson arrivals/s")
    ap.add_argument("--serving-slots", type=int, default=64)
    ap.add_argument("--serving-chunk", type=int, default=50)
    ap.add_argument("--serving-timeout", type=float, default=300.0)
    ap.add_argument("--serving-light-requests", type=int, default=16,
                    help="requests of a second serving run under the GPU's capacity (0 skips)")
    ap.add_argument("--serving-light-rate", type=float, default=2.0)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.report == "modes":
        return report_modes(args)
    if args.report == "kernels":
        return report_kernels(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
