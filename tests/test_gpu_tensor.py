"""GPU parity of the tensor-core schedule (tcgen05.mma on exact f16 integers, accumulators in
tensor memory): pass by pass against the FP64 oracle, bit-identical to the plain schedule, in
batches, with graphs and without, and refused where its exactness or geometry does not hold."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

E_REL = 1e-5
DE_REL = 1e-6


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


def _lockstep(s, tiles, n_sweeps, check_energy_every=0):
    for sweep in range(n_sweeps):
        s.optimize(1, stats=False)
        for i, ref in enumerate(tiles):
            dE, flags, couples = s.sweep_log(i)
            lg = ref.sweep(gpu_improving=(flags & 2) != 0)
            assert np.array_equal(couples, lg.couples), sweep
            valid = (lg.flags & 1) != 0
            err = np.abs(dE[valid].astype(np.float64) - lg.dE[valid])
            assert np.all(err <= DE_REL * lg.S[valid] + 1e-30), (sweep, err.max())
            assert np.array_equal(flags & 7, lg.flags & 7), sweep
        if check_energy_every and (sweep + 1) % check_energy_every == 0:
            e = s.energy()
            for i, ref in enumerate(tiles):
                assert abs(e[i] - ref.energy()) <= E_REL * ref.energy()
    for i, ref in enumerate(tiles):
        assert np.array_equal(s.counts(i), ref.k)
        assert np.array_equal(s.shifts()[i], ref.shifts_float())


# (W, H, N, T, pairs, radius, seed, passes)
LOCKSTEP = [
    (32, 32, 16, 64, 1, 6, 0, 30),      # the small published configuration
    (45, 37, 4, 100, 1, 6, 3, 12),      # ragged patches on both axes, P not a power of two
    (13, 13, 64, 1, 1, 6, 2, 12),       # narrowest torus for radius 6: one ragged patch
    (20, 17, 16, 40, 1, 6, 12, 12),     # the radius walk leaves a patch and re-enters it
    (24, 20, 64, 300, 2, 6, 5, 8),      # two pairs, ragged T
    (33, 47, 64, 256, 1, 8, 7, 8),      # radius 8: 29 classes, lists up to 768 pixels
    (40, 30, 32, 129, 1, 3, 4, 10),     # radius 3
    (48, 40, 64, 1024, 1, 6, 3, 4),     # T = 1024, 16 stages of 64 integrands
    (20, 20, 64, 4096, 1, 6, 1, 2),     # largest T of 8-bit counts: T N^2 = 2^24
    # 16-bit counts (N >= 128), centred f16 operands
    (32, 32, 256, 64, 1, 6, 3, 10),     # N = 256
    (45, 37, 128, 200, 2, 6, 4, 8),     # N = 128, two pairs, ragged patches and T
    (40, 40, 256, 512, 1, 6, 9, 4),     # T N^2 = 2^25: the last size with one accumulator round
    (36, 30, 256, 1024, 1, 6, 8, 4),    # two accumulator rounds of 8 stages (T N^2 = 2^26)
    (30, 28, 256, 1300, 1, 6, 13, 3),   # three rounds (8, 8, 5 stages), near the T limit of N
    (29, 27, 512, 320, 1, 6, 10, 3),    # N = 512: rounds of 2 stages (2, 2, 1)
    (31, 33, 512, 300, 2, 3, 11, 4),    # ragged T over rounds of 2 stages, two pairs, radius 3
    (33, 29, 512, 100, 1, 3, 2, 6),     # N = 512 (counts up to 512), radius 3
    (29, 31, 128, 70, 1, 8, 6, 6),      # radius 8 with 16-bit counts
    # the other radii (class tables of the generic epilogue paths)
    (27, 25, 16, 96, 1, 2, 14, 8),      # radius 2
    (30, 22, 64, 160, 1, 4, 15, 6),     # radius 4, ragged patches
    (36, 28, 256, 300, 1, 5, 16, 4),    # radius 5, 16-bit counts
    (40, 34, 32, 128, 2, 7, 17, 4),     # radius 7, two pairs
    (33, 35, 256, 1100, 1, 8, 18, 3),   # radius 8 with two accumulator rounds
]


@pytest.mark.parametrize("cfg", LOCKSTEP)
def test_lockstep_tensor_schedule(pkg, cfg):
    W, H, N, T, pairs, r, seed, passes = cfg
    s = pkg.Sampler(W, H, N, T, seed=seed, n_pairs=pairs, radius=r,
                    schedule=pkg.BN_SCHEDULE_TENSOR)
    assert s.get_schedule()["kind"] == pkg.BN_SCHEDULE_TENSOR
    tiles = [oracle.OracleTile(W, H, N, T, seed=seed, pair=i, radius=r) for i in range(pairs)]
    _lockstep(s, tiles, passes, check_energy_every=passes)
    s.close()


def test_lockstep_tensor_concurrent_mode(pkg):
    s = pkg.Sampler(32, 32, 16, 64, seed=5, mode=pkg.BN_MODE_CONCURRENT,
                    schedule=pkg.BN_SCHEDULE_TENSOR)
    ref = oracle.OracleTile(32, 32, 16, 64, seed=5, mode=oracle.MODE_CONCURRENT)
    _lockstep(s, [ref], 20)
    s.close()


def test_lockstep_tensor_literal_objective(pkg):
    s = pkg.Sampler(24, 20, 16, 48, seed=8, objective=pkg.BN_OBJECTIVE_LITERAL,
                    schedule=pkg.BN_SCHEDULE_TENSOR)
    ref = oracle.OracleTile(24, 20, 16, 48, seed=8, objective=oracle.OBJECTIVE_LITERAL)
    _lockstep(s, [ref], 20)
    s.close()


def _run(pkg, schedule, cfg, sweeps, graph_passes=None):
    W, H, N, T, pairs, seed = cfg
    s = pkg.Sampler(W, H, N, T, seed=seed, n_pairs=pairs, schedule=schedule)
    if graph_passes is not None:
        s.set_graph_passes(graph_passes)
    st = s.optimize(sweeps)
    out = (s.shifts(), [s.sweep_log(i) for i in range(pairs)], s.energy(), s.counts(0),
           (st.proposals, st.improving, st.committed, st.ties))
    s.close()
    return out


def _same(a, b):
    assert np.array_equal(a[0], b[0])
    for la, lb in zip(a[1], b[1]):
        for x, y in zip(la, lb):
            assert np.array_equal(x, y)
    assert np.array_equal(a[2], b[2])
    assert np.array_equal(a[3], b[3])
    assert a[4] == b[4]


@pytest.mark.parametrize("cfg", [(128, 128, 64, 1024, 1, 0), (64, 48, 64, 1024, 2, 21),
                                 (96, 80, 16, 256, 1, 4), (64, 64, 256, 512, 2, 5)])
def test_tensor_schedule_equals_plain(pkg, cfg):
    """Tiles, logs, energies, counts and statistics bit-identical to the plain schedule."""
    plain = _run(pkg, pkg.BN_SCHEDULE_PLAIN, cfg, 40)
    tens = _run(pkg, pkg.BN_SCHEDULE_TENSOR, cfg, 40)
    _same(tens, plain)


def test_tensor_graphs_do_not_change_results(pkg):
    cfg = (64, 64, 64, 512, 1, 9)
    a = _run(pkg, pkg.BN_SCHEDULE_TENSOR, cfg, 70, graph_passes=32)   # 2 replays + 6 direct
    b = _run(pkg, pkg.BN_SCHEDULE_TENSOR, cfg, 70, graph_passes=0)
    _same(a, b)


def test_tensor_batch_equals_each_alone(pkg):
    cfgs = [(32, 32, 16, 64, 1), (48, 40, 4, 256, 1), (64, 64, 64, 128, 2), (20, 36, 16, 1, 1),
            (128, 128, 64, 1024, 1), (45, 37, 64, 200, 1)]
    alone, mixed = [], []
    for W, H, N, T, pairs in cfgs:
        with pkg.Sampler(W, H, N, T, seed=W + H, n_pairs=pairs,
                         schedule=pkg.BN_SCHEDULE_PLAIN) as a:
            a.optimize(20, stats=False)
            alone.append((a.shifts(), a.energy()))
        mixed.append(pkg.Sampler(W, H, N, T, seed=W + H, n_pairs=pairs,
                                 schedule=pkg.BN_SCHEDULE_TENSOR))
    b = pkg.Batch(mixed)
    assert b.get_schedule()["kind"] == pkg.BN_SCHEDULE_TENSOR
    b.optimize(20, stats=False)
    for m, (sh, e) in zip(mixed, alone):
        assert np.array_equal(m.shifts(), sh)
        assert np.array_equal(m.energy(), e)
    b.close()
    for m in mixed:
        m.close()


def test_tensor_batch_of_mixed_widths_radii_and_rounds(pkg):
    """One tensor-core batch holding 8-bit and 16-bit problems (separately ordered patches),
    radii 3, 6 and 8, a problem in two accumulator rounds and a two-pair member, with per-member
    budgets: every member equals the plain schedule alone."""
    cfgs = [  # (W, H, N, T, pairs, radius, seed, passes)
        (48, 40, 16, 256, 1, 6, 1, 12), (40, 36, 256, 1024, 1, 6, 2, 9),
        (37, 29, 128, 200, 2, 3, 3, 14), (44, 30, 64, 512, 1, 8, 4, 7),
        (32, 32, 512, 300, 1, 6, 5, 10),
    ]
    mixed = [pkg.Sampler(W, H, N, T, seed=seed, n_pairs=p, radius=r,
                         schedule=pkg.BN_SCHEDULE_TENSOR)
             for W, H, N, T, p, r, seed, _ in cfgs]
    b = pkg.Batch(mixed)
    assert b.get_schedule()["kind"] == pkg.BN_SCHEDULE_TENSOR
    b.optimize_each([c[-1] for c in cfgs], stats=False)
    for m, (W, H, N, T, p, r, seed, n) in zip(mixed, cfgs):
        with pkg.Sampler(W, H, N, T, seed=seed, n_pairs=p, radius=r,
                         schedule=pkg.BN_SCHEDULE_PLAIN) as a:
            a.optimize(n, stats=False)
            assert np.array_equal(m.shifts(), a.shifts())
            assert np.array_equal(m.energy(), a.energy())
            assert m.get_state()[0] == a.get_state()[0]
    b.close()
    for m in mixed:
        m.close()


def test_tensor_batch_per_member_budgets(pkg):
    cfgs = [(32, 32, 16, 64, 1, 7), (64, 48, 64, 256, 1, 3), (40, 40, 64, 128, 2, 11)]
    budgets = [5, 17, 11]
    mixed = [pkg.Sampler(W, H, N, T, seed=seed, n_pairs=p, schedule=pkg.BN_SCHEDULE_TENSOR)
             for W, H, N, T, p, seed in cfgs]
    b = pkg.Batch(mixed)
    b.optimize_each(budgets, stats=False)
    for m, (W, H, N, T, p, seed), n in zip(mixed, cfgs, budgets):
        with pkg.Sampler(W, H, N, T, seed=seed, n_pairs=p, schedule=pkg.BN_SCHEDULE_PLAIN) as a:
            a.optimize(n, stats=False)
            assert np.array_equal(m.shifts(), a.shifts())
            assert m.get_state()[0] == a.get_state()[0]
    b.close()
    for m in mixed:
        m.close()


def test_switching_schedules_mid_run(pkg):
    """Plain -> tensor -> persistent -> tensor on one sampler equals plain throughout."""
    cfg = (64, 64, 64, 256, 1, 13)
    W, H, N, T, pairs, seed = cfg
    ref = _run(pkg, pkg.BN_SCHEDULE_PLAIN, cfg, 40)
    s = pkg.Sampler(W, H, N, T, seed=seed, schedule=pkg.BN_SCHEDULE_PLAIN)
    s.optimize(10, stats=False)
    for kind in (pkg.BN_SCHEDULE_TENSOR, pkg.BN_SCHEDULE_PERSISTENT, pkg.BN_SCHEDULE_TENSOR):
        s.set_schedule(kind)
        s.optimize(10, stats=False)
    assert np.array_equal(s.shifts(), ref[0])
    assert np.array_equal(s.energy(), ref[2])
    s.close()


@pytest.mark.parametrize("W,H,N,T,r", [(40, 40, 1024, 8, 6), (12, 40, 16, 64, 6),
                                       (40, 6, 16, 64, 3)])
def test_tensor_schedule_refused_outside_its_domain(pkg, W, H, N, T, r):
    """Counts of 1024 (N = 1024) and tiles narrower than 2 radius + 1 are refused."""
    from paper_2105_12620_gb300 import BnError
    with pytest.raises(BnError):
        pkg.Sampler(W, H, N, T, seed=1, radius=r, schedule=pkg.BN_SCHEDULE_TENSOR)
    s = pkg.Sampler(W, H, N, T, seed=1, radius=r)
    with pytest.raises(BnError):
        s.set_schedule(pkg.BN_SCHEDULE_TENSOR)
    # the sampler keeps a usable default schedule and still runs its passes
    assert s.get_schedule()["kind"] in (pkg.BN_SCHEDULE_PERSISTENT, pkg.BN_SCHEDULE_PLAIN)
    sw = s.get_state()[0]
    st = s.optimize(3)
    assert st.sweeps == 3 and s.get_state()[0] == sw + 3
    s.close()


def test_autotune_may_choose_the_tensor_schedule(pkg):
    """The tensor schedule is an autotuner candidate; whatever is chosen, results equal plain."""
    cfg = (128, 128, 64, 1024, 1, 2)
    W, H, N, T, pairs, seed = cfg
    s = pkg.Sampler(W, H, N, T, seed=seed)
    chosen = s.autotune(6)
    assert chosen["kind"] in (pkg.BN_SCHEDULE_TENSOR, pkg.BN_SCHEDULE_PERSISTENT)
    s.optimize(12, stats=False)
    ref = _run(pkg, pkg.BN_SCHEDULE_PLAIN, cfg, 12)
    assert np.array_equal(s.shifts(), ref[0])
    s.close()
