"""Pins of the oracle's random streams: Philox4x32-10 known answers, the candidate
permutation (Sec. 3.4) and the per-pass XOR scramble."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox(ctr, key)) == expect


def test_philox_counter_sensitivity():
    base = oracle.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(oracle.philox(c, [5, 6]), base)


@pytest.mark.parametrize("L", [2, 3, 5, 8, 12])
def test_permutation_is_bijection(L):
    perm = oracle.permutation(1234, 0, L)
    assert sorted(perm.tolist()) == list(range(1 << L))


def test_permutation_depends_on_seed_and_pair():
    p0 = oracle.permutation(7, 0, 8)
    assert not np.array_equal(p0, oracle.permutation(8, 0, 8))
    assert not np.array_equal(p0, oracle.permutation(7, 1, 8))


def test_permutation_is_uniform_on_small_domain():
    # the position of each value over many seeds should be uniform on [0, 8): chi-square
    L, n = 3, 4000
    counts = np.zeros((8, 8))
    for s in range(n):
        perm = oracle.permutation(s, 0, L)
        counts[np.arange(8), perm] += 1
    expected = n / 8
    chi2 = ((counts - expected) ** 2 / expected).sum()
    # 64 cells, 49 degrees of freedom: mean 49, sd ~10
    assert chi2 < 49 + 6 * 10


def test_sweep_couples_are_disjoint_and_xor_scrambled():
    L, M = 10, 128
    perm = oracle.permutation(3, 0, L)
    for s in range(5):
        c = oracle.sweep_couples(3, 0, s, L, M, perm)
        flat = c.reshape(-1)
        assert len(set(flat.tolist())) == 2 * M
        x = int(flat[0]) ^ int(perm[0])
        assert np.array_equal(flat, perm[: 2 * M] ^ x)
    # different passes use different XOR values
    xs = {int(oracle.sweep_couples(3, 0, s, L, M, perm)[0, 0]) ^ int(perm[0]) for s in range(20)}
    assert len(xs) > 10


def test_priority_key_orders_by_draw_then_index():
    k = [oracle.priority_key(9, 0, 4, j) for j in range(100)]
    assert len(set(k)) == 100
    for j, key in enumerate(k):
        assert key & 0xFFFFFFFF == 0xFFFFFFFF - j
        assert key >> 32 == oracle.philox([j, 4, 6, 0], [9, 0])[0]
