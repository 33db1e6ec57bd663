"""Seeded random configurations in lockstep with the oracle: tile sides 2..48 (ragged, non-square,
smaller than the stencil), N = 2..256 (8- and 16-bit counts), T = 1..300, radius 1..8, one or two
pairs, both commit rules, both objective directions, plain and persistent schedules.  Every draw
must match bit for bit (counts, couples, decisions outside the tie margin, shifts) and Eq. 1
within 1e-5."""
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


def draw_config(i):
    rng = np.random.default_rng(1000 + i)
    W = int(rng.integers(2, 49))
    H = int(rng.integers(2, 49))
    N = int(2 ** rng.integers(1, 9))
    radius = int(rng.integers(1, 9))
    # 24 T N^2 < 2^31 keeps the swap terms exact in int32
    tmax = min(300, (2 ** 31 - 1) // (24 * N * N))
    T = int(rng.integers(1, tmax + 1))
    pairs = int(rng.integers(1, 3))
    mode = int(rng.integers(0, 2))
    objective = int(rng.choice([-1, 1]))
    seed = int(rng.integers(0, 2 ** 40))
    # the persistent kernel needs radius 6 and tiles of at least 20 x 13
    persistent = radius == 6 and W >= 20 and H >= 13 and bool(rng.integers(0, 2))
    return dict(W=W, H=H, N=N, T=T, pairs=pairs, radius=radius, mode=mode, objective=objective,
                seed=seed, persistent=persistent)


# force a share of persistent-capable draws: radius 6 on larger tiles
def draw_persistent(i):
    c = draw_config(500 + i)
    rng = np.random.default_rng(7000 + i)
    c.update(W=int(rng.integers(20, 49)), H=int(rng.integers(13, 49)), radius=6, persistent=True)
    return c


CASES = [draw_config(i) for i in range(80)] + [draw_persistent(i) for i in range(24)]


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: "{W}x{H}_N{N}_T{T}_p{pairs}_r{radius}_m{mode}"
                         "_o{objective}_{sched}".format(sched="pers" if c["persistent"] else "plain",
                                                        **c))
def test_random_configuration_in_lockstep(pkg, cfg):
    kind = pkg.BN_SCHEDULE_PERSISTENT if cfg["persistent"] else pkg.BN_SCHEDULE_PLAIN
    s = pkg.Sampler(cfg["W"], cfg["H"], cfg["N"], cfg["T"], seed=cfg["seed"], n_pairs=cfg["pairs"],
                    radius=cfg["radius"], mode=cfg["mode"], objective=cfg["objective"],
                    schedule=kind)
    assert s.get_schedule()["kind"] == kind
    refs = [oracle.OracleTile(cfg["W"], cfg["H"], cfg["N"], cfg["T"], seed=cfg["seed"], pair=i,
                              radius=cfg["radius"], mode=cfg["mode"], objective=cfg["objective"])
            for i in range(cfg["pairs"])]
    for i, ref in enumerate(refs):
        assert np.array_equal(s.counts(i), ref.k)
    e = s.energy()
    for i, ref in enumerate(refs):
        want = ref.energy()
        assert abs(e[i] - want) <= E_REL * want + 1e-12
    for _ in range(16):
        s.optimize(1, stats=False)
        for i, ref in enumerate(refs):
            dE, flags, couples = s.sweep_log(i)
            lg = ref.sweep(gpu_improving=(flags & 2) != 0)
            assert np.array_equal(couples, lg.couples)
            valid = (lg.flags & 1) != 0
            err = np.abs(dE[valid].astype(np.float64) - lg.dE[valid])
            assert np.all(err <= DE_REL * lg.S[valid] + 1e-30)
            assert np.array_equal(flags & 7, lg.flags & 7)
    e = s.energy()
    sh = s.shifts()
    for i, ref in enumerate(refs):
        want = ref.energy()
        assert abs(e[i] - want) <= E_REL * want + 1e-12
        assert np.array_equal(s.counts(i), ref.k)
        assert np.array_equal(sh[i], ref.shifts_float())
    s.close()
