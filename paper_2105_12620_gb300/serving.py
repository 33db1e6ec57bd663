"""Load generator for the serving loop: a Poisson stream of sampler-generation requests, played
against a ``Server`` in real time, with latency percentiles, queue depth and throughput.

Request mix (one request = one tile to build and optimise): square tiles whose side is
log-uniform in [32, 512] (non-powers of two included), N drawn from {16, 64, 256}, T = 1024
Heavisides, one or two pairs of dimensions (2-D or 4-D), a pass budget uniform in [500, 5000].
The host logic here (drawing the stream, summarising the results) needs no GPU.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np


@dataclass
class Request:
    arrival: float     # seconds after the start of the run
    width: int
    height: int
    n_points: int
    n_integrands: int
    n_pairs: int
    n_sweeps: int
    seed: int


def draw_requests(n: int, rate_hz: float = 200.0, seed: int = 0, side=(32, 512),
                  n_points=(16, 64, 256), n_integrands: int = 1024, sweeps=(500, 5000),
                  pairs=(1, 2)) -> list[Request]:
    """n requests with exponential inter-arrival gaps of mean 1 / rate_hz (a Poisson stream)."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, n)) if n else np.zeros(0)
    sides = np.rint(np.exp(rng.uniform(math.log(side[0]), math.log(side[1]), n))).astype(int)
    ns = rng.choice(np.asarray(n_points), n)
    budgets = rng.integers(sweeps[0], sweeps[1] + 1, n)
    npairs = rng.choice(np.asarray(pairs), n)
    seeds = rng.integers(1, 1 << 62, n)
    return [Request(float(arrivals[i]), int(sides[i]), int(sides[i]), int(ns[i]), n_integrands,
                    int(npairs[i]), int(budgets[i]), int(seeds[i])) for i in range(n)]


def couples_per_pass(width: int, height: int) -> int:
    """Couples proposed per pass with the default setting: 2^ceil(log2 P) / 8, at least one."""
    P = width * height
    L = (P - 1).bit_length()
    return max(1, (1 << L) // 8)


def offered_proposals(reqs: list[Request]) -> int:
    """Upper bound of the proposals the stream asks for (couples x pairs x passes); couples whose
    candidate index falls beyond P in the padded range are not evaluated."""
    return sum(couples_per_pass(r.width, r.height) * r.n_pairs * r.n_sweeps for r in reqs)


def latency_percentiles(lat, wait) -> dict:
    """p50 / p99 of the per-request latencies (submit to done) and queueing delays (submit to
    admit), numpy's linear interpolation between order statistics; None for no requests."""
    lat, wait = np.asarray(lat, dtype=np.float64), np.asarray(wait, dtype=np.float64)
    pct = (lambda a, q: float(np.percentile(a, q)) if len(a) else None)
    return {"p50_latency_s": pct(lat, 50), "p99_latency_s": pct(lat, 99),
            "mean_latency_s": float(lat.mean()) if len(lat) else None,
            "p50_queue_s": pct(wait, 50), "p99_queue_s": pct(wait, 99)}


def summarize(reqs: list[Request], results: dict, makespan_s: float, proposals: int,
              depth_samples: list[tuple[int, int]]) -> dict:
    """Latency percentiles (submit to done, server clock), queueing delay, rates; the raw
    per-request latencies and delays ride along under "latencies_s" and "queue_s" so that
    several streams can be pooled."""
    lat = np.array([results[i].t_done - results[i].t_submit for i in range(len(reqs))])
    wait = np.array([results[i].t_admit - results[i].t_submit for i in range(len(reqs))])
    ok = sum(1 for r in results.values() if r.status == 0)
    span_arrivals = reqs[-1].arrival if reqs else 0.0
    depth = np.array([d for d, _ in depth_samples]) if depth_samples else np.zeros(1)
    active = np.array([a for _, a in depth_samples]) if depth_samples else np.zeros(1)
    return {
        "requests": len(reqs), "completed": ok,
        **latency_percentiles(lat, wait),
        "latencies_s": [float(v) for v in lat], "queue_s": [float(v) for v in wait],
        "offered_req_per_s": len(reqs) / span_arrivals if span_arrivals > 0 else None,
        "served_req_per_s": ok / makespan_s if makespan_s > 0 else None,
        "proposals_per_s": proposals / makespan_s if makespan_s > 0 else None,
        "offered_proposals_per_s": (offered_proposals(reqs) / span_arrivals
                                    if span_arrivals > 0 else None),
        "makespan_s": makespan_s,
        "max_queue_depth": int(depth.max()), "mean_resident": float(active.mean()),
    }


def run_load(server, reqs: list[Request], timeout_s: float = 600.0,
             poll_s: float = 0.0005) -> dict:
    """Submit each request at its arrival time, collect every result, and summarise."""
    results: dict[int, object] = {}
    depth: list[tuple[int, int]] = []
    proposals0 = server.stats()["proposals"]
    t0 = time.perf_counter()
    i = 0
    last_sample = -1.0
    while len(results) < len(reqs):
        now = time.perf_counter() - t0
        if now > timeout_s:
            raise TimeoutError(f"{len(results)} of {len(reqs)} requests done after {now:.0f} s")
        while i < len(reqs) and reqs[i].arrival <= now:
            r = reqs[i]
            server.submit(r.width, r.height, r.n_points, r.n_integrands, r.n_sweeps, seed=r.seed,
                          n_pairs=r.n_pairs, user_tag=i)
            i += 1
        for res in server.poll():
            results[res.user_tag] = res
            if res.status == 0:
                server.take_shifts(res)
        if now - last_sample >= 0.05:
            st = server.stats()
            depth.append((st["pending"], st["active"]))
            last_sample = now
        time.sleep(poll_s)
    makespan = time.perf_counter() - t0
    proposals = server.stats()["proposals"] - proposals0
    return summarize(reqs, results, makespan, proposals, depth)
