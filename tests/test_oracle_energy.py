"""Pins of the loss (Eq. 1) and of the energy change of a swap (Sec. 2, Sec. 3.4)."""
import math

import numpy as np
import pytest

import oracle
from tests._independent import energy_all_pairs, stencil_offsets

SIGMA, R = 2.1, 6


def _rand_counts(P, T, N, seed):
    return np.random.default_rng(seed).integers(0, N + 1, size=(P, T)).astype(np.int32)


@pytest.mark.parametrize("W,H,r", [(4, 4, 6), (5, 3, 6), (8, 8, 6), (6, 7, 2), (16, 16, 6),
                                   (9, 12, 3)])
def test_energy_matches_all_pairs_bruteforce(W, H, r):
    N, T = 16, 5
    k = _rand_counts(W * H, T, N, W * 100 + H)
    E, _ = oracle.energy(W, H, N, k, SIGMA, r)
    Eb = energy_all_pairs(W, H, N, k, SIGMA, r)
    assert abs(E - Eb) <= 1e-12 * abs(Eb)


def test_small_tile_counts_each_neighbour_once():
    # on a 4x4 torus every other pixel is within distance 6: 15 neighbours, all distinct
    N, T = 4, 1
    k = np.zeros((16, 1), np.int32)
    k[0, 0] = 1
    E, cls = oracle.energy(4, 4, N, k, SIGMA, R)
    # pixel 0 differs from each of its 15 neighbours by 1: 2 * sum_q w(d2(0,q)) / N^2
    d2s = [min(dx, 4 - dx) ** 2 + min(dy, 4 - dy) ** 2 for dy in range(4) for dx in range(4)][1:]
    expect = 2 * sum(math.exp(-d / SIGMA**2) for d in d2s) / N**2
    assert abs(E - expect) < 1e-14
    assert cls.sum() == 30


def test_energy_zero_for_identical_pixels():
    k = np.tile(np.arange(7, dtype=np.int32), (32 * 32, 1))
    assert oracle.energy(32, 32, 16, k, SIGMA, R)[0] == 0.0


def test_energy_invariances():
    W, H, N, T = 24, 18, 16, 6
    k = _rand_counts(W * H, T, N, 1).reshape(H, W, T)
    E0 = oracle.energy(W, H, N, k.reshape(-1, T), SIGMA, R)[0]
    for img, (w, h) in [(np.roll(k, (5, -3), axis=(0, 1)), (W, H)),
                        (k[::-1], (W, H)), (k[:, ::-1], (W, H)),
                        (np.transpose(k, (1, 0, 2)), (H, W)),
                        (np.rot90(k, 1, axes=(0, 1)), (H, W))]:
        E = oracle.energy(w, h, N, np.ascontiguousarray(img).reshape(-1, T), SIGMA, R)[0]
        assert abs(E - E0) <= 1e-12 * E0


def test_checkerboard_closed_form():
    """Two alternating vectors A, B: every pixel sees the other colour at the offsets with odd
    dx + dy, so E = P |A - B|^2 / N^2 * sum_{odd offsets} exp(-d^2 / sigma^2)."""
    W, H, N = 20, 14, 64
    A = np.array([3, 60, 17, 0], np.int32)
    B = np.array([40, 2, 17, 64], np.int32)
    y, x = np.mgrid[0:H, 0:W]
    k = np.where(((x + y) % 2 == 0)[..., None], A, B).reshape(-1, 4).astype(np.int32)
    E = oracle.energy(W, H, N, k, SIGMA, R)[0]
    wsum = sum(math.exp(-(dx * dx + dy * dy) / SIGMA**2) for dx, dy in stencil_offsets(R)
               if (dx + dy) % 2)
    expect = W * H * float(((A - B) ** 2).sum()) / N**2 * wsum
    assert abs(E - expect) <= 1e-12 * expect


def test_stencil_classes_and_weight_sum():
    offs = stencil_offsets(R)
    assert len(offs) == 112
    mult = {}
    for dx, dy in offs:
        mult[dx * dx + dy * dy] = mult.get(dx * dx + dy * dy, 0) + 1
    assert [mult[c] for c in sorted(mult)] == [4, 4, 4, 8, 4, 4, 8, 8, 4, 8, 4, 8, 12, 8, 8, 4,
                                              8, 4]
    assert abs(sum(math.exp(-(dx * dx + dy * dy) / SIGMA**2) for dx, dy in offs) - 12.850) < 1e-3
    # the per-distance class sums returned by the oracle use exactly these classes
    k = _rand_counts(32 * 32, 3, 16, 3)
    _, cls = oracle.energy(32, 32, 16, k, SIGMA, R)
    assert set(np.nonzero(cls)[0].tolist()) <= set(mult)


def _swap(k, a, b):
    k2 = k.copy()
    k2[[a, b]] = k2[[b, a]]
    return k2


@pytest.mark.parametrize("W,H", [(8, 8), (32, 32), (13, 17), (4, 4)])
def test_delta_energy_equals_full_recomputation(W, H):
    N, T = 16, 7
    k = _rand_counts(W * H, T, N, W + H)
    E0, c0 = oracle.energy(W, H, N, k, SIGMA, R)
    rng = np.random.default_rng(0)
    P = W * H
    pairs = [(0, 1), (0, W), (1, W + 2)] + [tuple(rng.choice(P, 2, replace=False)) for _ in range(12)]
    for a, b in pairs:
        a, b = int(a), int(b)
        dE, dcls = oracle.delta_energy(W, H, N, k, SIGMA, R, a, b)
        E1, c1 = oracle.energy(W, H, N, _swap(k, a, b), SIGMA, R)
        assert abs(dE - (E1 - E0)) <= 1e-12 * max(E0, 1.0)
        for c in range(R * R + 1):
            expect = math.exp(-c / SIGMA**2) * (c1[c] - c0[c]) / N**2
            assert abs(dcls[c] - expect) <= 1e-12 * max(abs(expect), 1e-30)


def test_delta_energy_of_identical_vectors_is_zero():
    k = _rand_counts(256, 4, 16, 9)
    k[5] = k[100]
    assert oracle.delta_energy(16, 16, 16, k, SIGMA, R, 5, 100)[0] == 0.0
