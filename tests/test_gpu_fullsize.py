"""Full-size parity of the multi-dimensional (256 x 256, N = 256, two pairs x T = 512, int16
counts) and batched (96 mixed tiles) configurations, in the launch configuration the benchmark
uses (fused persistent batch, autotuned schedule).

What the oracle computes in full here: shifts, integrands, permutation, the counts (in a pool of
spawned processes), Eq. 1 and two lockstep passes at 256 x 256; sampled tiles of the 96-tile
batch in lockstep.  What is checked by properties: after hundreds of passes the count vectors and
shifts are permutations of the initial ones, Eq. 1 never moved the wrong way, and the fused
persistent batch equals the plain schedule run alone."""
import copy
import os

import numpy as np
import pytest

import oracle
from paper_2105_12620_gb300 import workloads

pytestmark = pytest.mark.gpu

E_REL = 1e-5
DE_REL = 1e-6
WORKERS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_12620_gb300 import build
    build.build()
    import paper_2105_12620_gb300 as p
    p.load()
    return p


def _lockstep_pass(s, pair, ref):
    dE, flags, couples = s.sweep_log(pair)
    lg = ref.sweep(gpu_improving=(flags & 2) != 0)
    assert np.array_equal(couples, lg.couples)
    valid = (lg.flags & 1) != 0
    err = np.abs(dE[valid].astype(np.float64) - lg.dE[valid])
    assert np.all(err <= DE_REL * lg.S[valid] + 1e-30)
    assert np.array_equal(flags & 7, lg.flags & 7)


def _sorted_rows(a):
    return a[np.lexsort(a.T[::-1])]


@pytest.fixture(scope="module")
def multidim_refs():
    """The oracle's two pairs of the 256 x 256 configuration, computed once for the module."""
    cfg = workloads.c3()[0]
    W, H, N, T = cfg.width, cfg.height, cfg.n_points, cfg.n_integrands
    return [oracle.OracleTile(W, H, N, T, seed=0, pair=i, workers=WORKERS) for i in range(2)]


@pytest.mark.parametrize("schedule", ["autotuned", "tensor"])
def test_multidim_configuration_full_size(pkg, multidim_refs, schedule):
    cfg = workloads.c3()[0]
    W, H, N, T = cfg.width, cfg.height, cfg.n_points, cfg.n_integrands
    s = pkg.Sampler(W, H, N, T, seed=0, n_pairs=2)
    if schedule == "tensor":  # 16-bit counts as centred f16 operands of tcgen05.mma
        s.set_schedule(pkg.BN_SCHEDULE_TENSOR)
        assert s.get_schedule()["kind"] == pkg.BN_SCHEDULE_TENSOR
    else:
        s.autotune(10)
    refs = copy.deepcopy(multidim_refs)
    e = s.energy()
    k0 = []
    for i, ref in enumerate(refs):
        k = s.counts(i)
        assert np.array_equal(k, ref.k)
        k0.append(k)
        want = ref.energy()
        assert abs(e[i] - want) <= E_REL * want
        assert np.array_equal(s.permutation(i), ref.perm)
    assert np.array_equal(s.shifts(), np.stack([r.shifts_float() for r in refs]))
    for _ in range(2):
        s.optimize(1, stats=False)
        for i, ref in enumerate(refs):
            _lockstep_pass(s, i, ref)
    e2 = s.energy()
    for i, ref in enumerate(refs):
        want = ref.energy()
        assert abs(e2[i] - want) <= E_REL * want
        assert np.array_equal(s.counts(i), ref.k)
    # hundreds of passes more: permutations of the initial state, Eq. 1 only ever raised
    last = e2
    for _ in range(3):
        s.optimize(100, stats=False)
        cur = s.energy()
        assert np.all(cur >= last * (1 - E_REL))
        last = cur
    sh0 = np.stack([r.U / 2.0**32 for r in refs]).astype(np.float32)
    sh = s.shifts().reshape(2, -1, 2)
    for i in range(2):
        assert np.array_equal(_sorted_rows(sh[i]), _sorted_rows(sh0[i]))
        assert np.array_equal(_sorted_rows(s.counts(i)), _sorted_rows(k0[i]))
    # the same 302 passes on the plain schedule, alone
    with pkg.Sampler(W, H, N, T, seed=0, n_pairs=2, schedule=pkg.BN_SCHEDULE_PLAIN) as p:
        p.optimize(302, stats=False)
        assert np.array_equal(p.shifts(), s.shifts())
    s.close()


def test_batched_configuration_full_size(pkg):
    tiles = workloads.c4()
    samplers = [pkg.Sampler(t.width, t.height, t.n_points, t.n_integrands, seed=100 + i)
                for i, t in enumerate(tiles)]
    b = pkg.Batch(samplers)
    b.autotune(10)
    # lockstep a sample of the batch: the smallest tiles of each (N, T) and one 128 x 128
    picks = {}
    for i, t in enumerate(tiles):
        key = (t.n_points, t.n_integrands)
        if t.width <= 64 and key not in picks:
            picks[key] = i
    picks["big"] = next(i for i, t in enumerate(tiles) if t.width == 128 and t.n_integrands == 256)
    refs = {i: oracle.OracleTile(tiles[i].width, tiles[i].height, tiles[i].n_points,
                                 tiles[i].n_integrands, seed=100 + i, workers=WORKERS)
            for i in picks.values()}
    for i, ref in refs.items():
        assert np.array_equal(samplers[i].counts(0), ref.k)
    for _ in range(3):
        b.optimize(1, stats=False)
        for i, ref in refs.items():
            _lockstep_pass(samplers[i], 0, ref)
    for i, ref in refs.items():
        want = ref.energy()
        assert abs(samplers[i].energy()[0] - want) <= E_REL * want
    b.optimize(150, stats=False)
    for i in list(refs)[:4]:
        t = tiles[i]
        with pkg.Sampler(t.width, t.height, t.n_points, t.n_integrands, seed=100 + i,
                         schedule=pkg.BN_SCHEDULE_PLAIN) as a:
            a.optimize(153, stats=False)
            assert np.array_equal(a.shifts(), samplers[i].shifts())
    b.close()
    for s in samplers:
        s.close()
