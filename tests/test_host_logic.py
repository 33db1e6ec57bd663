"""Host-side logic that needs no GPU: the serving request stream and its summary, the bench's
per-rank seeds and clock parsing, and the multi-rank reductions (world size 2 over gloo)."""
import math
import os
import socket
from types import SimpleNamespace

import numpy as np
import pytest

import bench
from paper_2105_12620_gb300 import serving as srv


def test_request_stream_is_seeded_and_in_range():
    a = srv.draw_requests(500, 200.0, seed=3)
    b = srv.draw_requests(500, 200.0, seed=3)
    assert a == b
    assert a != srv.draw_requests(500, 200.0, seed=4)
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0)
    for r in a:
        assert 32 <= r.width == r.height <= 512
        assert r.n_points in (16, 64, 256) and r.n_integrands == 1024
        assert 500 <= r.n_sweeps <= 5000 and r.n_pairs in (1, 2)
        # every request is a valid configuration: 24 T N^2 < 2^31
        assert 24 * r.n_integrands * r.n_points ** 2 < 2 ** 31


def test_request_stream_distribution():
    n = 40000
    reqs = srv.draw_requests(n, 200.0, seed=1)
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert abs(gaps.mean() - 1 / 200.0) < 0.03 / 200.0           # Poisson rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.03             # exponential gaps: CV = 1
    side = np.array([r.width for r in reqs], float)
    # log-uniform on [32, 512]: half of the mass below sqrt(32 * 512) = 128
    assert abs((side <= 128).mean() - 0.5) < 0.02
    assert abs(np.mean([r.n_sweeps for r in reqs]) - 2750) < 30
    for v in (16, 64, 256):
        assert abs(np.mean([r.n_points == v for r in reqs]) - 1 / 3) < 0.02


def test_couples_per_pass_matches_the_padded_rule():
    import oracle
    for w, h in ((2, 2), (3, 2), (4, 4), (45, 37), (128, 128), (100, 7)):
        t = oracle.OracleTile(w, h, 4, 1, seed=0)
        assert srv.couples_per_pass(w, h) == t.M
    assert srv.couples_per_pass(128, 128) == 2048
    assert srv.couples_per_pass(129, 128) == 4096


def test_summary_percentiles_and_rates():
    reqs = [srv.Request(0.1 * i, 32, 32, 16, 1024, 1, 500, i) for i in range(101)]
    res = {i: SimpleNamespace(status=0, t_submit=0.1 * i, t_admit=0.1 * i + 0.01 * i,
                              t_done=0.1 * i + 1.0 + 0.01 * i) for i in range(101)}
    s = srv.summarize(reqs, res, makespan_s=20.0, proposals=4_000_000,
                      depth_samples=[(3, 5), (0, 7)])
    assert s["completed"] == 101
    assert math.isclose(s["p50_latency_s"], 1.5)
    assert math.isclose(s["p99_latency_s"], 1.0 + 0.99)
    assert math.isclose(s["p50_queue_s"], 0.5)
    assert math.isclose(s["offered_req_per_s"], 101 / 10.0)
    assert math.isclose(s["served_req_per_s"], 101 / 20.0)
    assert math.isclose(s["proposals_per_s"], 200_000.0)
    assert s["max_queue_depth"] == 3 and s["mean_resident"] == 6.0


def test_tile_seeds_are_distinct_across_ranks_steps_and_tiles():
    seen = set()
    for rank in range(8):
        for step in range(40):
            for tile in range(32):
                seen.add(bench.tile_seed(rank, step, tile, 32))
    assert len(seen) == 8 * 40 * 32


def test_parse_clocks():
    text = "\n".join([
        "0, 1965 MHz, 2070 MHz, 900 W, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 950, 0x4, Not Active, Not Active, Not Active, Active",
        "1, 600, 2070, 100, 0x0, Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 950, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    c = bench.parse_clocks(text, 0)
    assert c["sm_mhz"] == 1980 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    assert "hw_slowdown" in bench.parse_clocks(text, 1)["reasons"]
    assert bench.parse_clocks("", 0)["samples"] == 0


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank step times: the job's time is the slowest rank's
        t = bench.all_reduce_list([10.0 + rank, 20.0 - rank], dist, "cpu", "max")
        work = bench.all_reduce_list([100.0 * (rank + 1)], dist, "cpu", "sum")
        # uneven streams: rank 0 served latencies 0..99 s, rank 1 100..249 s (queue = 1/10)
        lat = [float(v) for v in (range(100) if rank == 0 else range(100, 250))]
        summ = {"p50_latency_s": -1.0, "p99_latency_s": -1.0, "p99_queue_s": -1.0,
                "makespan_s": 10.0 + 10.0 * rank, "proposals_per_s": 1e6,
                "completed": 5 + rank, "requests": len(lat), "latencies_s": lat,
                "queue_s": [v / 10 for v in lat]}
        merged = bench.merge_serving(summ, dist, "cpu")
        out.put((rank, t, work, merged))
    finally:
        dist.destroy_process_group()


def test_rank_reductions_world_size_two_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, work, merged in got:
        assert t == [11.0, 20.0]
        assert work == [300.0]
        # percentiles of the pooled 0..249 (250 samples): order statistic 0.5 * 249 = 124.5
        # and 0.99 * 249 = 246.51, linearly interpolated; the larger per-rank p50 would be 174.5
        assert merged["p50_latency_s"] == pytest.approx(124.5)
        assert merged["p99_latency_s"] == pytest.approx(246.51)
        assert merged["p99_queue_s"] == pytest.approx(24.651)
        assert merged["latency_samples"] == 250 and merged["requests"] == 250
        assert "latencies_s" not in merged and "queue_s" not in merged
        assert merged["makespan_s"] == 20.0
        # rank 0: 1e6/s over 10 s, rank 1: 1e6/s over 20 s -> 3e7 proposals in 20 s
        assert merged["proposals_per_s"] == pytest.approx(1.5e6)
        assert merged["completed"] == 11
        assert merged["served_req_per_s"] == pytest.approx(11 / 20.0)


def test_single_rank_serving_summary_keeps_its_percentiles():
    from paper_2105_12620_gb300 import serving as srv
    lat = [0.5, 0.1, 0.3, 0.2, 0.4]
    pct = srv.latency_percentiles(lat, [0.0] * 5)
    assert pct["p50_latency_s"] == pytest.approx(0.3)
    # order statistic 0.99 * 4 = 3.96 of the sorted 0.1 .. 0.5: 0.4 + 0.96 * 0.1
    assert pct["p99_latency_s"] == pytest.approx(0.496)
    assert srv.latency_percentiles([], [])["p99_latency_s"] is None
    summ = {**pct, "latencies_s": lat, "queue_s": [0.0] * 5, "makespan_s": 1.0,
            "completed": 5, "requests": 5, "proposals_per_s": 1.0}
    merged = bench.merge_serving(summ, None, "cpu")
    assert merged["p50_latency_s"] == pct["p50_latency_s"]
    assert merged["latency_samples"] == 5 and "latencies_s" not in merged


def test_workload_definitions():
    from paper_2105_12620_gb300 import workloads as wl
    c4 = wl.c4()
    assert len(c4) == 96 and c4 == wl.c4()
    assert {t.width for t in c4} == {32, 64, 128, 256}
    assert {t.n_points for t in c4} == {4, 16, 64} and {t.n_integrands for t in c4} == {256, 1024}
    assert all(t.width == t.height and t.sweeps == 2000 and t.n_pairs == 1 for t in c4)
    c3 = wl.c3()[0]
    assert (c3.width, c3.n_points, c3.n_integrands, c3.n_pairs, c3.sweeps) == (256, 256, 512, 2,
                                                                               4000)
    assert c3.couples() == 8192 and wl.c2()[0].couples() == 2048 and wl.c1()[0].couples() == 128
    assert wl.c2()[0].proposals() == 2048 * 2000
    # every workload is a valid configuration: 24 T N^2 < 2^31
    for t in c4 + [c3] + wl.c2() + wl.c1():
        assert 24 * t.n_integrands * t.n_points ** 2 < 2 ** 31


def test_measured_peak_reads_the_driver_file_or_falls_back(tmp_path, monkeypatch):
    val, how = bench.measured_peak("bf16_tflops")
    path = os.path.join(os.path.dirname(os.path.abspath(bench.__file__)), "MEASURED_PEAKS.json")
    if os.path.exists(path):
        import json
        assert how == "of measured" and val == float(json.load(open(path))["bf16_tflops"])
    else:
        assert how == "of fallback" and val == 1900.0
    # an unreadable or incomplete file falls back to the recipe's figures
    monkeypatch.setattr(bench.os.path, "dirname", lambda _p: str(tmp_path))
    assert bench.measured_peak("hbm_gbs") == (6800.0, "of fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 7000}')
    assert bench.measured_peak("hbm_gbs") == (7000.0, "of measured")
    assert bench.measured_peak("bf16_tflops") == (1900.0, "of fallback")


def test_schedule_description_of_the_json_line():
    t = bench.schedule_desc({"kind": 3, "shape": (0, 0, 0, 0), "tsplit": 0})
    assert t["kind"] == "tensor" and "block" not in t and t["chosen_by"] == "autotuner"
    p = bench.schedule_desc({"kind": 2, "shape": (8, 8, 256, 4), "tsplit": 1,
                             "chosen_by": "command line"})
    assert p == {"kind": "persistent", "block": [8, 8], "threads": 256, "tsplit": 1,
                 "chosen_by": "command line"}
    assert bench.schedule_desc({"kind": 1, "shape": (0, 0, 0, 0), "tsplit": 0})["kind"] == "plain"


def test_kernel_roofline_of_the_tensor_stencil():
    """The roofline object of the bench line: kept f16 FLOPs over the stencil's event time, the
    algorithmic count bytes, and the DRAM traffic of one launch scaled from the capture."""
    import argparse
    from paper_2105_12620_gb300 import workloads as wl
    specs = wl.c2(64)
    sweeps, split = specs[0].sweeps, 2
    launches, total_ms = split * sweeps, split * sweeps * 0.432
    ktimes = {"stencil_tensor": (launches, total_ms), "lists_tensor": (launches, 0.138 * launches)}
    args = argparse.Namespace(workload="c2")
    pkg = argparse.Namespace(BN_SCHEDULE_PERSISTENT=2)
    r = bench.kernel_roofline(ktimes, specs, split, sweeps, args, {"kind": 3}, pkg)
    P, T = 128 * 128, 1024
    kept_macs = 64 * (sweeps * P // 8) * 2 * 112 * T * split      # proposals x 2 sides x 112 x T
    secs = total_ms / 1000
    assert r["kernel"] == "stencil_tensor" and r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(2 * kept_macs / secs / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["avg_launch_ms"] == pytest.approx(0.432)
    assert r["share"] == pytest.approx(0.432 / (0.432 + 0.138))
    # one launch per pass at 64 tiles: the per-tile-pass bytes of the capture times 64
    assert r["traffic"] == pytest.approx(bench.TC_TRAFFIC_PER_TILE_PASS * 64)
    count_bytes = 64 * P * T * sweeps * split
    assert r["hbm"]["achieved"] == pytest.approx(count_bytes / secs / 1e9)
    # another workload: no capture to scale from
    r3 = bench.kernel_roofline(ktimes, specs, split, sweeps, argparse.Namespace(workload="c4"),
                               {"kind": 3}, pkg)
    assert r3["traffic"] is None
