"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Bit-exact: integrands, permutation, shifts, lattice points, counts, couples and commit decisions
(the oracle follows the GPU only on couples whose |dL| lies inside the 1e-6 relative tie margin).
Floating point: Eq. 1 within 1e-5 relative; per-couple dL within 1e-6 of the sum of absolute
per-distance terms (the fp32 compensated weighted sum is accurate to a few 2^-24 of that sum).
"""
import numpy as np
import pytest

import oracle
from oracle import FLAG_TIE

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


CONFIGS = [
    # (W, H, N, T, pairs, radius, seed)
    (32, 32, 16, 64, 1, 6, 0),        # the small published configuration
    (45, 37, 4, 100, 1, 6, 3),        # ragged tile (P not a power of two), ragged T
    (16, 16, 256, 300, 2, 6, 5),      # 16-bit counts, two pairs (4-D)
    (13, 13, 64, 1, 1, 6, 2),         # smallest tile with a full stencil, T = 1
    (4, 4, 2, 7, 1, 6, 9),            # tiny torus: every other pixel is a neighbour
    (9, 6, 32, 33, 1, 3, 4),          # other radius, non-square
    (64, 32, 128, 130, 1, 6, 11),     # N = 128 (16-bit), ragged T
    (2, 2, 8, 5, 1, 6, 1),            # smallest torus: one couple per pass, every swap a tie
    (3, 2, 16, 9, 1, 2, 6),           # P = 6 < 8 padded to 8: invalid couples occur
]


def _tiles(cfg):
    W, H, N, T, pairs, r, seed = cfg
    return [oracle.OracleTile(W, H, N, T, seed=seed, pair=i, radius=r) for i in range(pairs)]


def _sampler(pkg, cfg, **kw):
    W, H, N, T, pairs, r, seed = cfg
    return pkg.Sampler(W, H, N, T, seed=seed, n_pairs=pairs, radius=r, **kw)


@pytest.mark.parametrize("cfg", CONFIGS)
def test_initialisation_bit_exact(pkg, cfg):
    s = _sampler(pkg, cfg)
    for i, ref in enumerate(_tiles(cfg)):
        assert s.info.generator_g == ref.g
        a, b, C = s.integrands(i)
        assert np.array_equal(a, ref.a) and np.array_equal(b, ref.b) and np.array_equal(C, ref.C)
        assert np.array_equal(s.permutation(i), ref.perm)
        assert np.array_equal(s.counts(i), ref.k)
        assert np.array_equal(s.shifts()[i], ref.shifts_float())
        for pix in (0, ref.P - 1, ref.P // 3):
            x, y = oracle.points(ref.N, ref.g, *(ref.U[pix] / 2**32))
            pts = s.points(pix, i).astype(np.float64)
            assert np.array_equal(pts[:, 0], x) and np.array_equal(pts[:, 1], y)
    s.close()


@pytest.mark.parametrize("cfg", CONFIGS)
def test_energy_within_tolerance(pkg, cfg):
    s = _sampler(pkg, cfg)
    e = s.energy()
    for i, ref in enumerate(_tiles(cfg)):
        E = ref.energy()
        assert abs(e[i] - E) <= E_REL * E, (e[i], E)
    s.close()


def lockstep(s, tiles, n_sweeps, check_energy_every=0):
    """Run the GPU and the oracle pass by pass; return the number of tie-adopted couples."""
    ties = 0
    for sweep in range(n_sweeps):
        s.optimize(1, stats=False)
        for i, ref in enumerate(tiles):
            dE, flags, couples = s.sweep_log(i)
            lg = ref.sweep(gpu_improving=(flags & 2) != 0)
            assert np.array_equal(couples, lg.couples), sweep
            valid = (lg.flags & 1) != 0
            assert np.array_equal(flags & 1, lg.flags & 1)
            err = np.abs(dE[valid].astype(np.float64) - lg.dE[valid])
            assert np.all(err <= DE_REL * lg.S[valid] + 1e-30), (sweep, err.max())
            assert np.array_equal(flags & 7, lg.flags & 7), sweep
            ties += int(((lg.flags & FLAG_TIE) != 0).sum())
        if check_energy_every and (sweep + 1) % check_energy_every == 0:
            e = s.energy()
            for i, ref in enumerate(tiles):
                E = ref.energy()
                assert abs(e[i] - E) <= E_REL * E
    for i, ref in enumerate(tiles):
        assert np.array_equal(s.counts(i), ref.k)
        assert np.array_equal(s.shifts()[i], ref.shifts_float())
    return ties


def test_lockstep_small_configuration_200_passes(pkg):
    cfg = CONFIGS[0]
    s = _sampler(pkg, cfg)
    lockstep(s, _tiles(cfg), 200, check_energy_every=50)
    s.close()


@pytest.mark.parametrize("cfg", CONFIGS[1:])
def test_lockstep_edge_configurations(pkg, cfg):
    s = _sampler(pkg, cfg)
    lockstep(s, _tiles(cfg), 25, check_energy_every=25)
    s.close()


def test_lockstep_literal_objective(pkg):
    W, H, N, T = 24, 20, 16, 48
    s = pkg.Sampler(W, H, N, T, seed=8, objective=pkg.BN_OBJECTIVE_LITERAL)
    ref = oracle.OracleTile(W, H, N, T, seed=8, objective=oracle.OBJECTIVE_LITERAL)
    lockstep(s, [ref], 30)
    s.close()


def test_objective_monotone_on_gpu(pkg):
    s = pkg.Sampler(64, 64, 16, 128, seed=2)
    e = [s.energy()[0]]
    for _ in range(10):
        s.optimize(10, stats=False)
        e.append(s.energy()[0])
    # default objective raises Eq. 1 (tolerance: fp32 evaluation of the energy)
    assert all(e[i + 1] >= e[i] * (1 - 1e-6) for i in range(10))
    assert e[-1] > e[0]
    s.close()


def test_split_calls_equal_one_call(pkg):
    a = pkg.Sampler(40, 24, 16, 64, seed=3)
    b = pkg.Sampler(40, 24, 16, 64, seed=3)
    a.optimize(37, stats=False)
    a.optimize(1, stats=False)
    a.optimize(22, stats=False)
    b.optimize(60, stats=False)
    assert np.array_equal(a.shifts(), b.shifts())
    assert a.get_state()[0] == b.get_state()[0] == 60
    a.close()
    b.close()


def test_checkpoint_and_resume(pkg):
    a = pkg.Sampler(32, 32, 16, 64, seed=6, n_pairs=2)
    a.optimize(40, stats=False)
    sweep, sidx = a.get_state()
    c = pkg.Sampler(32, 32, 16, 64, seed=6, n_pairs=2)
    c.set_state(sweep, sidx)
    assert np.array_equal(c.counts(1), a.counts(1))
    a.optimize(30, stats=False)
    c.optimize(30, stats=False)
    assert np.array_equal(a.shifts(), c.shifts())
    a.close()
    c.close()


def test_stats_are_consistent_with_the_log(pkg):
    s = pkg.Sampler(32, 32, 16, 64, seed=0)
    st = s.optimize(1)
    dE, flags, couples = s.sweep_log()
    assert st.sweeps == 1
    assert st.proposals == int(((flags & 1) != 0).sum())
    assert st.improving == int(((flags & 2) != 0).sum())
    assert st.committed == int(((flags & 4) != 0).sum())
    assert st.ties == int(((flags & 8) != 0).sum())
    s.close()


def test_batch_equals_each_alone(pkg):
    cfgs = [(32, 32, 16, 64, 1), (48, 40, 4, 256, 1), (64, 64, 64, 128, 2), (20, 36, 16, 1, 1)]
    alone, mixed = [], []
    for W, H, N, T, pairs in cfgs:
        a = pkg.Sampler(W, H, N, T, seed=W + H, n_pairs=pairs)
        a.optimize(40, stats=False)
        alone.append(a.shifts())
        a.close()
        mixed.append(pkg.Sampler(W, H, N, T, seed=W + H, n_pairs=pairs))
    b = pkg.Batch(mixed)
    b.optimize(15, stats=False)
    b.optimize(25, stats=False)
    for m, ref in zip(mixed, alone):
        assert np.array_equal(m.shifts(), ref)
    b.close()
    for m in mixed:
        m.close()


def test_full_size_gpu_scale_configuration(pkg):
    """128 x 128, N = 64, T = 1024 (int8 counts): sampled pixels' counts recomputed one by one
    by the oracle, full Eq. 1, and three lockstep passes at full size."""
    W = H = 128
    s = pkg.Sampler(W, H, 64, 1024, seed=0)
    ref = oracle.OracleTile(W, H, 64, 1024, seed=0)
    assert np.array_equal(s.counts(), ref.k)
    E = ref.energy()
    assert abs(s.energy()[0] - E) <= E_REL * E
    lockstep(s, [ref], 3)
    s.close()


def test_lockstep_concurrent_mode(pkg):
    s = pkg.Sampler(32, 32, 16, 64, seed=5, mode=pkg.BN_MODE_CONCURRENT)
    ref = oracle.OracleTile(32, 32, 16, 64, seed=5, mode=oracle.MODE_CONCURRENT)
    lockstep(s, [ref], 40)
    s.close()


@pytest.mark.parametrize("cfg", [(32, 32, 16, 64, 1, 6, 0), (45, 37, 4, 100, 1, 6, 3),
                                 (24, 20, 256, 300, 2, 6, 5), (64, 32, 128, 130, 1, 6, 11),
                                 (20, 13, 16, 40, 1, 6, 12)])
def test_lockstep_persistent_schedule(pkg, cfg):
    s = _sampler(pkg, cfg, schedule=pkg.BN_SCHEDULE_PERSISTENT)
    assert s.get_schedule()["kind"] == pkg.BN_SCHEDULE_PERSISTENT
    lockstep(s, _tiles(cfg), 30 if cfg[0] == 32 else 12, check_energy_every=6)
    s.close()


def test_persistent_shape_falls_back_on_narrow_tiles(pkg):
    """A requested shape that does not fit the tiles gives way to the first one that does: a
    16-pixel-wide block needs tiles at least 16 + 2 r wide."""
    s = pkg.Sampler(24, 24, 16, 64, seed=1)
    s.set_schedule(pkg.BN_SCHEDULE_PERSISTENT, (16, 8, 512, 4), 1)
    sc = s.get_schedule()
    assert sc["kind"] == pkg.BN_SCHEDULE_PERSISTENT and sc["shape"] == (8, 8, 256, 4)
    s.close()


def test_persistent_lockstep_concurrent_mode(pkg):
    s = pkg.Sampler(32, 32, 16, 64, seed=5, mode=pkg.BN_MODE_CONCURRENT,
                    schedule=pkg.BN_SCHEDULE_PERSISTENT)
    ref = oracle.OracleTile(32, 32, 16, 64, seed=5, mode=oracle.MODE_CONCURRENT)
    lockstep(s, [ref], 30)
    s.close()


def _run_with(pkg, kind, shape, tsplit, cfg, sweeps):
    W, H, N, T, pairs, seed = cfg
    s = pkg.Sampler(W, H, N, T, seed=seed, n_pairs=pairs)
    s.set_schedule(kind, shape, tsplit)
    s.optimize(sweeps, stats=False)
    out = (s.shifts(), s.sweep_log(0), s.energy())
    s.close()
    return out


@pytest.mark.parametrize("cfg", [(64, 48, 64, 1024, 1, 21), (40, 40, 256, 200, 2, 4)])
def test_schedule_does_not_change_results(pkg, cfg):
    """Every instantiated CTA shape and chunk split of the persistent kernel, and the plain
    schedule, produce bit-identical tiles, logs and energies."""
    from paper_2105_12620_gb300._lib import PERSISTENT_SHAPES
    base = _run_with(pkg, pkg.BN_SCHEDULE_PLAIN, None, 0, cfg, 25)
    for shape in PERSISTENT_SHAPES:
        for tsplit in (1, 2, 4):
            got = _run_with(pkg, pkg.BN_SCHEDULE_PERSISTENT, shape, tsplit, cfg, 25)
            assert np.array_equal(got[0], base[0]), (shape, tsplit)
            for x, y in zip(got[1], base[1]):
                assert np.array_equal(x, y), (shape, tsplit)
            assert np.array_equal(got[2], base[2])


def test_persistent_batch_equals_each_alone(pkg):
    cfgs = [(32, 32, 16, 64, 1), (48, 40, 4, 256, 1), (64, 64, 64, 128, 2), (20, 36, 16, 1, 1),
            (128, 128, 64, 1024, 1), (40, 24, 256, 128, 1)]
    alone, mixed = [], []
    for W, H, N, T, pairs in cfgs:
        a = pkg.Sampler(W, H, N, T, seed=W + H, n_pairs=pairs, schedule=pkg.BN_SCHEDULE_PLAIN)
        a.optimize(30, stats=False)
        alone.append(a.shifts())
        a.close()
        mixed.append(pkg.Sampler(W, H, N, T, seed=W + H, n_pairs=pairs))
    b = pkg.Batch(mixed)
    assert b.get_schedule()["kind"] == pkg.BN_SCHEDULE_PERSISTENT
    b.optimize(11, stats=False)
    b.optimize(19, stats=False)
    for m, ref in zip(mixed, alone):
        assert np.array_equal(m.shifts(), ref)
    b.close()
    for m in mixed:
        m.close()


@pytest.mark.parametrize("kind", ["plain", "persistent"])
def test_batch_per_member_budgets(pkg, kind):
    """bn_batch_optimize_each: each member stops at its own pass budget inside the fused launch
    (zero included), and ends exactly where it would alone; its pass counter says so."""
    cfgs = [(32, 32, 16, 64, 1), (48, 40, 4, 256, 1), (64, 64, 64, 128, 2), (40, 24, 256, 128, 1)]
    budgets = [[7, 0, 13, 3], [5, 9, 0, 11]]
    sched = pkg.BN_SCHEDULE_PLAIN if kind == "plain" else pkg.BN_SCHEDULE_AUTO
    mixed = [pkg.Sampler(W, H, N, T, seed=W * 3 + H, n_pairs=p, schedule=sched)
             for W, H, N, T, p in cfgs]
    b = pkg.Batch(mixed)
    want = pkg.BN_SCHEDULE_PLAIN if kind == "plain" else pkg.BN_SCHEDULE_PERSISTENT
    assert b.get_schedule()["kind"] == want
    total = [0] * len(cfgs)
    for bud in budgets:
        b.optimize_each(bud, stats=False)
        total = [t + x for t, x in zip(total, bud)]
    for m, (W, H, N, T, p), n in zip(mixed, cfgs, total):
        assert m.get_state()[0] == n
        with pkg.Sampler(W, H, N, T, seed=W * 3 + H, n_pairs=p) as a:
            a.optimize(n, stats=False)
            assert np.array_equal(m.shifts(), a.shifts())
            assert np.array_equal(m.energy(), a.energy())
    b.close()
    for m in mixed:
        m.close()


def test_plain_graphs_do_not_change_results(pkg):
    """Plain schedule replayed from captured CUDA graphs (several graph sizes, pass counts that
    are not multiples of them) equals direct launches, alone and in a batch."""
    def run(graph, cfg, passes):
        W, H, N, T, pairs, seed = cfg
        s = pkg.Sampler(W, H, N, T, seed=seed, n_pairs=pairs, schedule=pkg.BN_SCHEDULE_PLAIN)
        s.set_graph_passes(graph)
        for n in passes:
            s.optimize(n, stats=False)
        out = (s.shifts(), s.sweep_log(0), s.energy(), s.get_state()[0])
        s.close()
        return out

    for cfg in [(32, 32, 16, 64, 1, 3), (45, 37, 128, 100, 2, 4), (9, 6, 8, 20, 1, 5)]:
        base = run(0, cfg, [75, 40])
        for graph in (1, 7, 32):
            got = run(graph, cfg, [75, 40])
            assert np.array_equal(got[0], base[0]) and np.array_equal(got[2], base[2])
            assert got[3] == base[3] == 115
            for x, y in zip(got[1], base[1]):
                assert np.array_equal(x, y)
    cfgs = [(32, 32, 16, 64, 1), (20, 36, 4, 256, 1), (10, 10, 64, 32, 2)]
    tiles = [pkg.Sampler(W, H, N, T, seed=W + H, n_pairs=p, schedule=pkg.BN_SCHEDULE_PLAIN)
             for W, H, N, T, p in cfgs]
    b = pkg.Batch(tiles)
    b.set_graph_passes(8)
    b.optimize(37, stats=False)
    b.optimize_each([20, 0, 9], stats=False)
    for t, (W, H, N, T, p), n in zip(tiles, cfgs, (57, 37, 46)):
        with pkg.Sampler(W, H, N, T, seed=W + H, n_pairs=p, schedule=pkg.BN_SCHEDULE_PLAIN) as a:
            a.set_graph_passes(0)
            a.optimize(n, stats=False)
            assert np.array_equal(t.shifts(), a.shifts())
    b.close()
    for t in tiles:
        t.close()


def test_autotune_leaves_state_alone_and_keeps_results(pkg):
    cfgs = [(48, 40, 16, 128, 1), (64, 64, 64, 256, 1), (40, 40, 256, 128, 2)]
    tiles = [pkg.Sampler(W, H, N, T, seed=W * 7 + H, n_pairs=p) for W, H, N, T, p in cfgs]
    for t in tiles:
        t.optimize(5, stats=False)
    before = [(t.shifts(), t.counts(0), t.get_state()[0]) for t in tiles]
    b = pkg.Batch(tiles)
    chosen = b.autotune(4)
    assert chosen["kind"] in (pkg.BN_SCHEDULE_PERSISTENT, pkg.BN_SCHEDULE_PLAIN,
                              pkg.BN_SCHEDULE_TENSOR)
    for t, (sh, k, sw) in zip(tiles, before):
        assert np.array_equal(t.shifts(), sh) and np.array_equal(t.counts(0), k)
        assert t.get_state()[0] == sw
    assert b.autotune(4) == chosen          # cached
    b.optimize(20, stats=False)
    refs = [pkg.Sampler(W, H, N, T, seed=W * 7 + H, n_pairs=p, schedule=pkg.BN_SCHEDULE_PLAIN)
            for W, H, N, T, p in cfgs]
    for r in refs:
        r.optimize(25, stats=False)
    for t, r in zip(tiles, refs):
        assert np.array_equal(t.shifts(), r.shifts())
        r.close()
    b.close()
    for t in tiles:
        t.close()


def test_bounded_waits_report_timeouts_and_the_context_survives(pkg):
    """The kernels' grid barrier and mbarrier waits give up after their clock budget and report
    it (no trap, no hang); afterwards the GPU context is still usable."""
    from paper_2105_12620_gb300 import _lib as L
    lib = L.load()
    for which in (0, 1):
        assert lib.bn_selftest_wait_timeout(which, 1 << 22) == L.BN_ERR_TIMEOUT
        assert "ran out" in lib.bn_last_error().decode()
    s = pkg.Sampler(32, 32, 16, 64, seed=1)
    st = s.optimize(3)
    assert st.sweeps == 3 and st.proposals > 0
    s.close()
