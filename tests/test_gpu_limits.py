"""Configurations at the limits of bn_config: N = 1024 (16-bit counts up to 1024), T = 4096, the
largest tile (P = 2^22), zero-pass calls, and the exact-arithmetic bound 24 T N^2 < 2^31."""
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


def _lockstep(s, refs, n):
    for _ in range(n):
        s.optimize(1, stats=False)
        for i, ref in enumerate(refs):
            dE, flags, couples = s.sweep_log(i)
            lg = ref.sweep(gpu_improving=(flags & 2) != 0)
            assert np.array_equal(couples, lg.couples)
            valid = (lg.flags & 1) != 0
            err = np.abs(dE[valid].astype(np.float64) - lg.dE[valid])
            assert np.all(err <= DE_REL * lg.S[valid] + 1e-30)
            assert np.array_equal(flags & 7, lg.flags & 7)


@pytest.mark.parametrize("W,H,N,T,seed", [
    (20, 16, 1024, 64, 1),     # largest N: 16-bit counts reach 1024; 24 T N^2 = 1.6e9 < 2^31
    (16, 13, 2, 4096, 2),      # largest T (32 chunks of 128 bytes per pixel)
    (24, 20, 256, 1365, 3),    # 24 T N^2 = 2 146 959 360, just below 2^31
])
def test_extreme_n_and_t_in_lockstep(pkg, W, H, N, T, seed):
    s = pkg.Sampler(W, H, N, T, seed=seed)
    ref = oracle.OracleTile(W, H, N, T, seed=seed)
    assert np.array_equal(s.counts(0), ref.k)
    want = ref.energy()
    assert abs(s.energy()[0] - want) <= E_REL * want
    _lockstep(s, [ref], 8)
    assert np.array_equal(s.shifts()[0], ref.shifts_float())
    s.close()


def test_exact_arithmetic_bound_is_enforced(pkg):
    from paper_2105_12620_gb300 import BnError
    with pytest.raises(BnError):
        pkg.Sampler(16, 16, 64, 21846, seed=1)     # 24 * 21846 * 64^2 >= 2^31 (and T > 4096)
    with pytest.raises(BnError):
        pkg.Sampler(16, 16, 1024, 90, seed=1)      # 24 * 90 * 1024^2 >= 2^31


def test_zero_passes_change_nothing(pkg):
    s = pkg.Sampler(32, 32, 16, 64, seed=4)
    sh, e, st = s.shifts(), s.energy(), s.get_state()[0]
    stats = s.optimize(0)
    assert stats.sweeps == 0 and stats.proposals == 0 and stats.committed == 0
    assert np.array_equal(s.shifts(), sh) and np.array_equal(s.energy(), e)
    assert s.get_state()[0] == st
    b = pkg.Batch([s])
    b.optimize(0, stats=False)
    b.optimize_each([0], stats=False)
    assert np.array_equal(s.shifts(), sh) and s.get_state()[0] == st
    b.close()
    s.close()


def test_largest_tile(pkg):
    """2048 x 2048 (P = 2^22, the largest tile): sampled pixels' counts recomputed by the oracle
    one by one, the shifts bit-exact, and after passes the shift and count multisets unchanged
    with Eq. 1 moved only the intended way."""
    W = H = 2048
    N, T = 16, 32
    s = pkg.Sampler(W, H, N, T, seed=5)
    U = oracle.shifts(5, 0, W * H)
    a, b, C = oracle.heaviside_bank(5, 0, T)
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(W * H, 512, replace=False))
    k = s.counts(0)
    assert np.array_equal(k[sample], oracle.counts(N, oracle.pick_g(N), U[sample], a, b, C))
    assert np.array_equal(s.shifts()[0].reshape(-1, 2), (U / 2.0**32).astype(np.float32))
    e0 = s.energy()[0]
    st = s.optimize(20)
    assert st.proposals == 20 * (W * H // 8) and st.committed > 0
    assert s.energy()[0] >= e0 * (1 - E_REL)
    sh = s.shifts()[0].reshape(-1, 2)
    order = lambda x: x[np.lexsort(x.T[::-1])]
    assert np.array_equal(order(sh), order((U / 2.0**32).astype(np.float32)))
    # count vectors: the same multiset (rows compared through a random 64-bit hash)
    w = rng.integers(1, 2**62, T, dtype=np.int64) | 1
    rows = lambda m: np.sort((m.astype(np.int64) * w).sum(axis=1))
    assert np.array_equal(rows(s.counts(0)), rows(k))
    s.close()
