"""Pins of the test-integrand map (Sec. 2, Fig. 1b): counts k_p[t] = sum_k f_t(s^k_p) of random
Heavisides f(x, y) = [a x + b y < c] over each pixel's shifted lattice."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests._independent import half_plane_area

TWO24 = 1 << 24


def _axis_count(N, u_fixed, theta: Fraction, below=True):
    """#{i : (u + i/N) mod 1 < theta} (or > theta), exact rationals: the 1-D projection of any
    shifted N-point rank-1 lattice with g odd is u0 + i/N, u0 = u mod 1/N."""
    u0 = Fraction(int(u_fixed), 1 << 32) % Fraction(1, N)
    pts = [u0 + Fraction(i, N) for i in range(N)]
    return sum(1 for v in pts if (v < theta if below else v > theta))


@pytest.mark.parametrize("N", [2, 16, 64, 256])
def test_axis_aligned_heavisides_closed_form(N):
    g = oracle.pick_g(N)
    rng = np.random.default_rng(5 + N)
    U = (rng.integers(0, 1 << 24, size=(12, 2)) << 8).astype(np.uint32)
    a = np.array([3, 0, -7, 0, 1 << 15, 0], np.int32)
    b = np.array([0, 5, 0, -2, 0, -(1 << 15)], np.int32)
    C = np.zeros(6, np.int64)
    thetas = [Fraction(int(x), TWO24) for x in rng.integers(1, TWO24, size=6)]
    for t in range(6):
        coef = int(a[t]) + int(b[t])  # one of them is zero
        # a x < C / 2^24  with C = coef * theta * 2^24 (exact integer)
        C[t] = int(coef * thetas[t] * TWO24)
    k = oracle.counts(N, g, U, a, b, C)
    for p in range(U.shape[0]):
        for t in range(6):
            coef = int(a[t]) + int(b[t])
            theta = Fraction(int(C[t]), TWO24) / coef
            u = U[p, 0] if a[t] != 0 else U[p, 1]
            expect = _axis_count(N, u, theta, below=coef > 0)
            assert k[p, t] == expect, (N, p, t)


def test_complementary_half_planes_sum_to_N():
    N = 64
    U = oracle.shifts(11, 0, 50)
    a, b, C = oracle.heaviside_bank(11, 0, 40)
    k1 = oracle.counts(N, 19, U, a, b, C)
    k2 = oracle.counts(N, 19, U, -a, -b, -C + 1)   # [v < C] + [-v < -C + 1] = [v<C] + [v>=C]
    assert np.all(k1 + k2 == N)


def test_counts_unbiased_against_exact_area():
    """A randomly shifted lattice estimates the integral without bias: the mean of k/N over
    many random shifts converges to the area of the half-plane inside the unit square."""
    N, nshift = 16, 6000
    U = oracle.shifts(99, 0, nshift)
    a, b, C = oracle.heaviside_bank(99, 0, 24)
    k = oracle.counts(N, oracle.pick_g(N), U, a, b, C) / N
    for t in range(24):
        area = half_plane_area(float(a[t]), float(b[t]), float(C[t]) / TWO24)
        mean = k[:, t].mean()
        se = max(k[:, t].std(ddof=1), 1e-3) / math.sqrt(nshift)
        assert abs(mean - area) < 5 * se + 1e-6, (t, mean, area)


def test_shift_by_a_lattice_vector_permutes_points():
    N, g = 64, 19
    U = oracle.shifts(5, 0, 30)
    a, b, C = oracle.heaviside_bank(5, 0, 32)
    k0 = oracle.counts(N, g, U, a, b, C)
    x, y = oracle.points(N, g, 0.0, 0.0)
    for kk in (1, 7, 33):
        lat = np.array([round(x[kk] * 2**32) % 2**32, round(y[kk] * 2**32) % 2**32], np.uint64)
        U2 = ((U.astype(np.uint64) + lat) % 2**32).astype(np.uint32)
        assert np.array_equal(oracle.counts(N, g, U2, a, b, C), k0)


def test_counts_range_and_integrand_bank():
    a, b, C = oracle.heaviside_bank(2021, 1, 4000)
    q = a.astype(np.int64) ** 2 + b.astype(np.int64) ** 2
    assert np.all(q > 0) and np.all(q <= 1 << 30)
    lo = np.minimum(a, 0).astype(np.int64) + np.minimum(b, 0)
    hi = np.maximum(a, 0).astype(np.int64) + np.maximum(b, 0)
    # the edge crosses the unit square
    assert np.all(C >= lo * TWO24) and np.all(C < hi * TWO24)
    # orientation uniform on the circle, offset uniform over the projection of the square
    ang = np.sort((np.arctan2(b, a) + math.pi) / (2 * math.pi))
    frac = np.sort((C - lo * TWO24) / ((hi - lo) * TWO24))
    n = len(ang)
    for v in (ang, frac):
        ks = np.max(np.abs(v - (np.arange(1, n + 1) - 0.5) / n))
        assert ks < 1.8 / math.sqrt(n)


def test_shifts_are_24_bit_uniform():
    U = oracle.shifts(7, 0, 20000)
    assert np.all(U & 0xFF == 0)
    u = np.sort(U[:, 0] / 2**32)
    n = len(u)
    assert np.max(np.abs(u - (np.arange(1, n + 1) - 0.5) / n)) < 1.8 / math.sqrt(n)
    assert not np.array_equal(oracle.shifts(7, 0, 64), oracle.shifts(7, 1, 64))


def test_parallel_counts_equal_serial_counts():
    N, g = 16, oracle.pick_g(16)
    U = oracle.shifts(3, 0, 37)
    a, b, C = oracle.heaviside_bank(3, 0, 21)
    assert np.array_equal(oracle.counts_parallel(N, g, U, a, b, C, 3),
                          oracle.counts(N, g, U, a, b, C))
