"""Pins of the main sequence (Sec. 3.2): rank-1 lattice s^k = mod(Phi(k) d, 1) with a Korobov
direction vector, scrambled by a toroidal shift mod(s^k + u_p, 1)."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_van_der_corput_first_values():
    expect = [0, 1 / 2, 1 / 4, 3 / 4, 1 / 8, 5 / 8, 3 / 8, 7 / 8, 1 / 16]
    assert [oracle.van_der_corput(k) for k in range(9)] == expect


def _min_pair_distance(N, g):
    # all pairs of lattice points, toroidal, in units of 1/N (independent of the oracle's
    # difference-to-origin shortcut)
    k = np.arange(N)
    x = k
    y = (k * g) % N
    dx = np.abs(x[:, None] - x[None, :])
    dy = np.abs(y[:, None] - y[None, :])
    dx = np.minimum(dx, N - dx)
    dy = np.minimum(dy, N - dy)
    d2 = dx * dx + dy * dy
    d2[k, k] = np.iinfo(np.int64).max
    return int(d2.min())


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64, 128, 256])
def test_korobov_search_matches_all_pairs_bruteforce(N):
    gs = [g for g in range(1, N) if np.gcd(g, N) == 1]
    d = {g: _min_pair_distance(N, g) for g in gs}
    for g in gs:
        assert oracle.korobov_min_dist2(N, g) == d[g]
    best = max(d.values())
    assert oracle.pick_g(N) == min(g for g in gs if d[g] == best)


def test_korobov_tie_sets():
    # g = 5, used by the paper's teaser, is one of the N = 16 optima
    for N, ties in [(4, {1, 3}), (16, {3, 5, 11, 13}), (64, {19, 27, 37, 45}),
                    (256, {71, 119, 137, 185})]:
        d = {g: oracle.korobov_min_dist2(N, g) for g in range(1, N, 2)}
        best = max(d.values())
        assert {g for g in d if d[g] == best} == ties


def _teaser():
    pts = {"green": {}, "red": {}}
    for line in open(os.path.join(GOLDEN, "teaser_fig1a_points.txt")):
        if line.startswith("#") or not line.strip():
            continue
        s, k, x, y = line.split()
        pts[s][int(k)] = (float(x), float(y))
    return pts


def test_teaser_points_fig1a():
    """Fig. 1a prints two shifted copies of a 16-point lattice.  Their x column is
    mod(u_x + Phi(k), 1) for all k (d_1 = 1); their y column follows g = 5 with u_y = 0.5625 on
    the entries k in {1,3,5,6,7,9,11,13,14,15}; the other six y entries are garbled in print."""
    reliable_y = {1, 3, 5, 6, 7, 9, 11, 13, 14, 15}
    for name, pts in _teaser().items():
        ux = pts[0][0]
        x, y = oracle.points(16, 5, ux, 0.5625)
        for k in range(16):
            assert abs(x[k] - pts[k][0]) < 2e-6, (name, k)
            if k in reliable_y:
                assert abs(y[k] - pts[k][1]) < 2e-6, (name, k)


@pytest.mark.parametrize("N", [4, 16, 64, 256])
def test_projections_are_equally_spaced(N):
    g = oracle.pick_g(N)
    rng = np.random.default_rng(N)
    for _ in range(5):
        U = rng.integers(0, 1 << 24, size=2) << 8
        x, y = oracle.points(N, g, U[0] / 2**32, U[1] / 2**32)
        for v, u in ((x, U[0]), (y, U[1])):
            vs = np.sort(v)
            # exact: every coordinate is u + i/N mod 1 for a distinct i
            fr = sorted(Fraction(float(a)).limit_denominator(1 << 40) for a in vs)
            base = Fraction(int(u), 1 << 32) % Fraction(1, N)
            assert fr == [base + Fraction(i, N) for i in range(N)]


def test_unshifted_lattice_is_a_group():
    N, g = 64, 19
    x, y = oracle.points(N, g, 0.0, 0.0)
    pts = {(round(a * N), round(b * N)) for a, b in zip(x, y)}
    assert len(pts) == N
    for p in pts:
        for q in pts:
            assert ((p[0] - q[0]) % N, (p[1] - q[1]) % N) in pts


def test_screen_samples_wrap_pairs_and_padding():
    """Renderer lookup: the tile repeats over the screen, dimensions come in pairs, each pair
    from its own tile, and an odd dimension count drops the padding coordinate."""
    W, H, N = 5, 3, 16
    g = oracle.pick_g(N)
    U = [oracle.shifts(2, 0, W * H), oracle.shifts(2, 1, W * H)]
    s = oracle.screen_samples(N, g, U, W, H, -7, 4, 12, 5, 3, 9, 3)
    assert s.shape == (5, 12, 9, 3)
    # screen pixel (x, y) and (x + W, y - H) read the same tile pixel
    assert np.array_equal(s[:, :7], s[:, 5:12])
    assert np.array_equal(s[0], oracle.screen_samples(N, g, U, W, H, -7, 4 + H, 12, 1, 3, 9, 3)[0])
    # each pair's N samples of a pixel are its shifted lattice: every 1-D projection is the
    # N-point grid j / N shifted by the pixel's u (mod 1)
    full = oracle.screen_samples(N, g, U, W, H, 0, 0, W, H, 0, N, 4)
    for p in range(W * H):
        y, x = divmod(p, W)
        for pair in range(2):
            for c in range(2):
                u = U[pair][p, c] / 2**32
                v = np.sort((full[y, x, :, 2 * pair + c] - u) % 1.0)
                assert np.allclose(v, np.arange(N) / N, atol=1e-12)
    # the odd dimension count keeps the first coordinate of the last pair only
    assert np.array_equal(s[..., 2], oracle.screen_samples(N, g, U, W, H, -7, 4, 12, 5, 3, 9,
                                                           4)[..., 2])
