"""Serving loop (continuous batching) on the GPU: every request's outcome equals the same request
run alone through a Sampler, whatever else is resident, however the passes are chunked and
whenever it is admitted; admission respects the slot and memory limits; cancellation."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2105_12620_gb300 import BnError, Sampler, Server  # noqa: E402
from paper_2105_12620_gb300 import _lib as L  # noqa: E402

# (width, height, N, T, n_pairs, passes, seed): non-power-of-two tiles, 8- and 16-bit counts
MIX_PERSISTENT = [
    (24, 20, 16, 64, 1, 23, 11),
    (32, 32, 64, 256, 2, 40, 12),
    (40, 28, 32, 128, 1, 31, 13),
    (20, 20, 256, 64, 2, 12, 14),
    (48, 36, 128, 192, 1, 19, 15),
    (33, 47, 64, 1024, 1, 9, 16),
]
# a 16 x 16 tile is too small for the persistent kernel: batches holding it run plain
MIX_PLAIN = [
    (16, 16, 128, 128, 1, 17, 21),
    (24, 24, 16, 64, 2, 26, 22),
    (13, 29, 32, 96, 1, 11, 23),
]


# tensor-core capable requests (sides >= 13, N <= 512) beside ones that are not: N = 1024
# (counts of 1024 leave the f16 operand's exact range) and a 12 x 40 tile (narrower than the
# stencil)
MIX_TENSOR = [
    (64, 48, 64, 1024, 1, 21, 31),
    (37, 29, 16, 256, 2, 33, 32),
    (96, 80, 256, 512, 1, 12, 33),
    (20, 52, 128, 1000, 1, 17, 34),
    (48, 44, 256, 1024, 2, 9, 35),    # two accumulator rounds
]
MIX_NOT_TENSOR = [
    (40, 40, 1024, 16, 1, 14, 41),
    (12, 40, 16, 64, 1, 19, 42),
]


def alone(w, h, n, t, pairs, passes, seed):
    with Sampler(w, h, n, t, seed=seed, n_pairs=pairs) as s:
        s.optimize(passes, stats=False)
        return np.asarray(s.energy()), s.shifts()


def run_server(mix, max_slots, chunk, late=(), policy=L.BN_SERVE_TENSOR_TUNED):
    with Server(max_slots=max_slots, sweeps_per_chunk=chunk, tensor_policy=policy) as sv:
        ids = {}
        for k, (w, h, n, t, pairs, passes, seed) in enumerate(mix):
            ids[sv.submit(w, h, n, t, passes, seed=seed, n_pairs=pairs, user_tag=k)] = k
        if late:  # arrive while the first wave is on the GPU
            t0 = time.time()
            while sv.stats()["chunks"] < 1 and time.time() - t0 < 60:
                time.sleep(0.001)
            for k, (w, h, n, t, pairs, passes, seed) in enumerate(late, start=len(mix)):
                ids[sv.submit(w, h, n, t, passes, seed=seed, n_pairs=pairs, user_tag=k)] = k
        sv.drain(300.0)
        results = sv.poll(1024)
        out = {}
        for r in results:
            assert r.status == L.BN_OK
            assert ids[r.request_id] == r.user_tag
            out[r.user_tag] = (np.asarray(r.energy), sv.take_shifts(r), r)
        stats = sv.stats()
    return out, stats


@pytest.mark.parametrize("mix,max_slots,chunk", [
    (MIX_PERSISTENT, 3, 7),
    (MIX_PERSISTENT, 16, 5),
    (MIX_PLAIN, 2, 6),
    (MIX_PERSISTENT[:3] + MIX_PLAIN[:2], 4, 9),
])
def test_each_result_equals_the_request_alone(mix, max_slots, chunk):
    out, stats = run_server(mix, max_slots, chunk)
    assert stats["completed"] == len(mix) and stats["failed"] == 0
    assert stats["pending"] == 0 and stats["active"] == 0 and stats["memory_in_use"] == 0
    for k, cfg in enumerate(mix):
        e_ref, sh_ref = alone(*cfg)
        e, sh, r = out[k]
        np.testing.assert_array_equal(sh, sh_ref)
        np.testing.assert_array_equal(e, e_ref)
        assert r.t_submit <= r.t_admit <= r.t_done


@pytest.mark.parametrize("policy", [L.BN_SERVE_TENSOR_ALWAYS, L.BN_SERVE_TENSOR_TUNED,
                                    L.BN_SERVE_TENSOR_NEVER], ids=["always", "tuned", "never"])
def test_tensor_batch_results_equal_the_request_alone(policy):
    """Requests on the tensor-core batch, beside requests the schedule refuses, give the results
    of the same requests run alone (on the default schedule)."""
    mix = MIX_TENSOR + MIX_NOT_TENSOR
    out, stats = run_server(mix, 4, 8, policy=policy)
    assert stats["completed"] == len(mix) and stats["failed"] == 0
    if policy == L.BN_SERVE_TENSOR_ALWAYS:
        assert stats["tensor_chunks"] > 0 and stats["tunes"] == 0
    if policy == L.BN_SERVE_TENSOR_NEVER:
        assert stats["tensor_chunks"] == 0 and stats["tunes"] == 0
    if policy == L.BN_SERVE_TENSOR_TUNED:
        # one trial per signature of a capable request, none for the others
        assert stats["tunes"] == len(MIX_TENSOR)
    for k, cfg in enumerate(mix):
        e_ref, sh_ref = alone(*cfg)
        e, sh, _ = out[k]
        np.testing.assert_array_equal(sh, sh_ref)
        np.testing.assert_array_equal(e, e_ref)


def test_tensor_batch_with_mid_flight_arrivals():
    first, late = MIX_TENSOR[:2] + MIX_NOT_TENSOR[:1], MIX_TENSOR[2:] + MIX_NOT_TENSOR[1:]
    out, stats = run_server(first, 8, 5, late=late, policy=L.BN_SERVE_TENSOR_ALWAYS)
    assert stats["completed"] == len(first) + len(late) and stats["tensor_chunks"] > 0
    for k, cfg in enumerate(first + late):
        e_ref, sh_ref = alone(*cfg)
        np.testing.assert_array_equal(out[k][1], sh_ref)
        np.testing.assert_array_equal(out[k][0], e_ref)


def test_requests_arriving_mid_flight_are_admitted_and_exact():
    first, late = MIX_PERSISTENT[:3], MIX_PERSISTENT[3:]
    out, stats = run_server(first, 8, 4, late=late)
    assert stats["completed"] == len(first) + len(late)
    for k, cfg in enumerate(first + late):
        e_ref, sh_ref = alone(*cfg)
        np.testing.assert_array_equal(out[k][1], sh_ref)
        np.testing.assert_array_equal(out[k][0], e_ref)


def test_proposal_count_matches_the_budgets():
    mix = MIX_PERSISTENT[:4]
    _, stats = run_server(mix, 2, 6)
    expect = 0
    for (w, h, n, t, pairs, passes, seed) in mix:
        with Sampler(w, h, n, t, seed=seed, n_pairs=pairs) as s:
            expect += s.info.couples * pairs * passes
    assert stats["proposals"] == expect


def test_memory_budget_serialises_admission_and_rejects_oversize():
    cfg = (64, 64, 64, 1024, 1, 30, 31)
    with Sampler(*cfg[:4], seed=cfg[6]) as s:
        bytes_one = s.info.device_bytes
    # room for one such request at a time
    with Server(max_slots=8, sweeps_per_chunk=10,
                memory_budget_bytes=int(bytes_one * 1.6) + (1 << 20)) as sv:
        for k in range(3):
            sv.submit(*cfg[:4], cfg[5], seed=cfg[6] + k, user_tag=k)
        with pytest.raises(BnError) as ei:
            sv.submit(256, 256, 64, 1024, 10)
        assert ei.value.code == L.BN_ERR_BUSY
        sv.drain(300.0)
        res = sorted(sv.poll(16), key=lambda r: r.t_admit)
        st = sv.stats()
    assert st["rejected"] == 1 and st["completed"] == 3
    assert [r.status for r in res] == [L.BN_OK] * 3
    for a, b in zip(res, res[1:]):
        assert b.t_admit >= a.t_done  # never two resident at once
    for r in res:
        with Sampler(*cfg[:4], seed=cfg[6] + r.user_tag) as s:
            s.optimize(cfg[5], stats=False)
            np.testing.assert_array_equal(np.asarray(r.energy), np.asarray(s.energy()))


def test_cancel_pending_and_resident():
    with Server(max_slots=1, sweeps_per_chunk=5) as sv:
        a = sv.submit(64, 64, 64, 512, 400, seed=1, user_tag=0)
        b = sv.submit(32, 32, 16, 64, 10, seed=2, user_tag=1)
        c = sv.submit(32, 32, 16, 64, 10, seed=3, user_tag=2)
        sv.cancel(b)
        t0 = time.time()
        while sv.stats()["chunks"] < 2 and time.time() - t0 < 60:
            time.sleep(0.001)
        sv.cancel(a)
        sv.drain(120.0)
        res = {r.request_id: r for r in sv.poll(16)}
        st = sv.stats()
        assert res[a].status == L.BN_ERR_BAD_STATE and res[b].status == L.BN_ERR_BAD_STATE
        assert res[c].status == L.BN_OK
        assert st["cancelled"] == 2 and st["completed"] == 1 and st["memory_in_use"] == 0
        with pytest.raises(BnError):
            sv.cancel(12345)


def test_concurrent_submitters_and_random_cancellations():
    """Four threads submit at once while the loop runs; a random third of the requests is
    cancelled.  Every request gets exactly one result; completed ones equal the request alone."""
    import threading
    rng = np.random.default_rng(5)
    cfgs = [(int(rng.choice([24, 32, 40])), int(rng.choice([20, 32])), int(rng.choice([16, 64])),
             64, 1, int(rng.integers(5, 40)), 200 + i) for i in range(24)]
    with Server(max_slots=6, sweeps_per_chunk=4) as sv:
        ids = [None] * len(cfgs)

        def submit(part):
            for k in part:
                w, h, n, t, pairs, passes, seed = cfgs[k]
                ids[k] = sv.submit(w, h, n, t, passes, seed=seed, n_pairs=pairs, user_tag=k)

        threads = [threading.Thread(target=submit, args=(range(q, len(cfgs), 4),))
                   for q in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        cancel = set(int(k) for k in rng.choice(len(cfgs), 8, replace=False))
        for k in cancel:
            try:
                sv.cancel(ids[k])
            except BnError:
                pass   # already finished
        sv.drain(300.0)
        res = {r.user_tag: r for r in sv.poll(1024)}
        assert sorted(res) == list(range(len(cfgs)))
        st = sv.stats()
        assert st["completed"] + st["cancelled"] == len(cfgs) and st["memory_in_use"] == 0
        for k, r in res.items():
            if r.status == L.BN_OK:
                e_ref, sh_ref = alone(*cfgs[k])
                np.testing.assert_array_equal(sv.take_shifts(r), sh_ref)
                np.testing.assert_array_equal(np.asarray(r.energy), e_ref)
            else:
                assert r.status == L.BN_ERR_BAD_STATE and k in cancel


def test_destroy_with_work_in_flight_returns():
    sv = Server(max_slots=4, sweeps_per_chunk=10)
    for k in range(6):
        sv.submit(64, 64, 64, 512, 2000, seed=k)
    time.sleep(0.2)
    t0 = time.time()
    sv.close()                      # drops queued and resident requests after the current chunk
    assert time.time() - t0 < 30.0
