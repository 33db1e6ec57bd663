"""Pins of the criterion oracle (Sec. 3.3 filtered-error RMSE, Sec. 3.5 smooth integrands)
against closed forms, brute force and a second, independent filter."""
import math

import numpy as np
import pytest

import oracle
from oracle import criterion as cr
from tests._independent import half_plane_area, torus_gaussian_blur


def test_heaviside_area_matches_polygon_clipping():
    a, b, C = oracle.heaviside_bank(5, 0, 400)
    for t in range(400):
        want = half_plane_area(float(a[t]), float(b[t]), C[t] / 16777216.0)
        assert abs(cr.heaviside_area(int(a[t]), int(b[t]), int(C[t])) - want) < 1e-12


@pytest.mark.parametrize("a,b,c,want", [
    (1, 0, 0.3, 0.3), (-1, 0, -0.3, 0.7), (0, 2, 1.0, 0.5), (0, -4, -1.0, 0.75),
    (1, 1, 1.0, 0.5), (1, 1, 0.5, 0.125), (1, 1, 1.5, 0.875), (1, -1, 0.0, 0.5),
    (3, 1, 10.0, 1.0), (3, 1, -1.0, 0.0),
])
def test_heaviside_area_closed_forms(a, b, c, want):
    # c is quantised to the 2^-24 grid of C: the area moves by at most 2^-24 / |normal|
    assert abs(cr.heaviside_area(a, b, round(c * 16777216)) - want) < 2e-7


def test_bump_integral_matches_a_fine_midpoint_rule():
    n = 1200
    xs = (np.arange(n) + 0.5) / n
    for cx, cy, s in [(0.5, 0.5, 0.1), (0.05, 0.9, 0.3), (0.99, 0.01, 0.5), (0.3, 0.7, 0.05)]:
        fx = np.exp(-(xs - cx) ** 2 / (2 * s * s))
        fy = np.exp(-(xs - cy) ** 2 / (2 * s * s))
        num = fx.mean() * fy.mean()
        assert abs(cr.bump_integral(cx, cy, s) - num) < 1e-6 * max(num, 1e-3)


def test_bump_bank_ranges_and_seeding():
    bank = cr.bump_bank(3, 0, 2000)
    assert np.all((bank[:, :2] >= 0) & (bank[:, :2] < 1))
    assert np.all((bank[:, 2] >= 0.05) & (bank[:, 2] < 0.5))
    assert abs(bank[:, 0].mean() - 0.5) < 0.02 and abs(bank[:, 2].mean() - 0.275) < 0.01
    assert not np.array_equal(bank, cr.bump_bank(3, 1, 2000))
    assert np.array_equal(bank, cr.bump_bank(3, 0, 2000))


def test_periodic_gaussian_weights():
    for n, s in [(32, 0.25), (32, 2.0), (7, 3.0), (128, 20.0), (5, 40.0)]:
        w = cr.periodic_gaussian(n, s)
        assert abs(w.sum() - 1.0) < 1e-14
        assert np.allclose(w[1:], w[1:][::-1], rtol=1e-13, atol=1e-300)  # symmetric: w[d]=w[n-d]
    # a wide tile: the sampled Gaussian itself
    w = cr.periodic_gaussian(256, 1.5)
    d = np.minimum(np.arange(256), 256 - np.arange(256))
    g = np.exp(-d**2 / (2 * 1.5**2))
    assert np.allclose(w, g / g.sum(), rtol=1e-12, atol=1e-300)
    # far wider than the tile: the filter becomes the mean
    assert np.allclose(cr.periodic_gaussian(6, 500.0), 1 / 6, rtol=1e-9)
    assert cr.periodic_gaussian(9, 0.0)[0] == 1.0


def test_blur_equals_direct_periodic_convolution():
    rng = np.random.default_rng(0)
    err = rng.normal(size=(3, 5, 4))
    for s in (0.25, 0.8, 3.0):
        wx, wy = cr.periodic_gaussian(4, s), cr.periodic_gaussian(5, s)
        want = np.zeros_like(err)
        for t in range(3):
            for y in range(5):
                for x in range(4):
                    want[t, y, x] = sum(wy[dy] * wx[dx] * err[t, (y + dy) % 5, (x + dx) % 4]
                                        for dy in range(5) for dx in range(4))
        assert np.allclose(cr.blur(err, s), want, rtol=1e-12, atol=1e-14)
    assert np.allclose(cr.blur(err, 0.0), err, atol=1e-15)


def test_blur_agrees_with_the_continuous_fourier_filter():
    # sampling the Gaussian aliases its spectrum by about exp(-2 pi^2 sigma^2 (1 - f)^2) at
    # frequency f <= 1/2: below 1e-19 for sigma >= 3, where the two filters must agree
    rng = np.random.default_rng(1)
    err = rng.normal(size=(2, 48, 40))
    for s in (3.0, 4.0, 11.0):
        ind = np.moveaxis(torus_gaussian_blur(np.moveaxis(err, 0, -1), s), -1, 0)
        assert np.allclose(cr.blur(err, s), ind, rtol=1e-9, atol=1e-12)


def test_rmse_of_constant_and_white_errors():
    const = np.full((2, 16, 12), -0.25)
    assert np.allclose(cr.rmse(const, [0.0, 0.5, 3.0, 30.0]), 0.25, rtol=1e-12)
    rng = np.random.default_rng(2)
    err = rng.normal(0, 0.1, size=(64, 64, 64))
    for s in (1.0, 3.0):
        wx = cr.periodic_gaussian(64, s)
        expect = 0.1 * math.sqrt((wx**2).sum() ** 2)    # Parseval: variance x sum of w^2
        assert abs(cr.rmse(err, [s])[0] / expect - 1) < 0.05


def test_bump_errors_follow_the_lattice_estimate():
    N, g = 64, oracle.pick_g(64)
    U = oracle.shifts(4, 0, 6)
    bank = cr.bump_bank(4, 0, 3)
    e = cr.bump_errors(N, g, U, bank, 3, 2)
    for p in range(6):
        x, y = oracle.points(N, g, U[p, 0] / 2**32, U[p, 1] / 2**32)
        for t in range(3):
            cx, cy, s = bank[t]
            est = np.mean(np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s * s)))
            assert abs(e[t, p // 3, p % 3] - (est - cr.bump_integral(cx, cy, s))) < 1e-15
    # a rank-1 lattice integrates smooth bumps well: errors far below plain MC at N = 256
    e = cr.bump_errors(256, oracle.pick_g(256), oracle.shifts(4, 0, 16), cr.bump_bank(4, 0, 8),
                       4, 4)
    assert np.abs(e).max() < 5e-3


def test_optimised_tile_lowers_filtered_error_for_both_integrand_kinds():
    """Sec. 3.3 / 3.5: after the optimisation the filtered error of the Heaviside estimates and
    of smooth bumps (never seen by the optimiser) is lower than for the initial random tile."""
    W = H = 24
    t = oracle.OracleTile(W, H, 16, 64, seed=3)
    bank = cr.bump_bank(99, 0, 24)
    sig = [1.0, 2.0, 4.0]

    def measure():
        eh = cr.heaviside_errors(t.k, t.N, t.a, t.b, t.C, W, H)
        eb = cr.bump_errors(t.N, t.g, t.U[t.sidx], bank, W, H)
        return cr.rmse(eh, sig), cr.rmse(eb, sig)

    h0, b0 = measure()
    for _ in range(150):
        t.sweep()
    h1, b1 = measure()
    assert np.all(h1 < 0.8 * h0), (h0, h1)
    assert np.all(b1 < 0.9 * b0), (b0, b1)
    # no filter: the per-pixel error is the same multiset (a swap moves estimates around)
    assert abs(cr.rmse(cr.heaviside_errors(t.k, t.N, t.a, t.b, t.C, W, H), [0.0])[0]
               - cr.rmse(cr.heaviside_errors(oracle.OracleTile(W, H, 16, 64, seed=3).k, 16,
                                             t.a, t.b, t.C, W, H), [0.0])[0]) < 1e-12


# ---------------------------------------------------------------------------------------------
# error spectrum (Fig. 1b)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("fx,fy,W,H,want", [
    (0, 0, 32, 32, 0), (1, 0, 32, 32, 1), (3, 4, 32, 32, 5), (1, 1, 32, 32, 1),
    (2, 2, 32, 32, 3), (16, 16, 32, 32, 23), (-7, 2, 32, 32, 7),
    # 2:1 tile: (1, 0) lies exactly half way, rho L = 1/2, and rounds up
    (1, 0, 64, 32, 1), (0, 1, 64, 32, 1), (3, 0, 64, 32, 2), (32, 16, 64, 32, 23),
])
def test_ring_of_known_values(fx, fy, W, H, want):
    assert cr.ring_of(fx, fy, W, H) == want


def test_ring_of_agrees_with_the_float_radius_off_the_half_way_points():
    rng = np.random.default_rng(8)
    for _ in range(2000):
        W, H = (int(v) for v in rng.integers(2, 300, 2))
        fx, fy = int(rng.integers(-W // 2, W // 2 + 1)), int(rng.integers(-H // 2, H // 2 + 1))
        r = math.hypot(fx / W, fy / H) * min(W, H)
        if abs(r - math.floor(r) - 0.5) > 1e-9:
            assert cr.ring_of(fx, fy, W, H) == math.floor(r + 0.5)


def test_spectrum_against_the_dft_by_definition():
    """np.fft against the DFT sum written out, on small tiles (even and odd sides)."""
    rng = np.random.default_rng(3)
    for W, H in ((6, 4), (5, 3), (7, 7)):
        err = rng.normal(size=(3, H, W))
        power, counts = cr.error_spectrum(err)
        ring, n = cr.rings(W, H)
        want = np.zeros(n)
        for t in range(3):
            for v in range(H):
                for u in range(W):
                    F = sum(err[t, y, x] * complex(math.cos(2 * math.pi * (u * x / W + v * y / H)),
                                                   -math.sin(2 * math.pi * (u * x / W + v * y / H)))
                            for y in range(H) for x in range(W))
                    want[ring[v, u]] += abs(F) ** 2 / (W * H)
        want /= 3 * counts
        assert np.allclose(power, want, rtol=1e-10, atol=1e-14)
        assert counts.sum() == W * H


def test_spectrum_parseval_and_a_single_cosine():
    rng = np.random.default_rng(4)
    err = rng.normal(0, 0.3, size=(5, 24, 40))
    power, counts = cr.error_spectrum(err)
    # Parseval: the ring sums add up to the mean squared error per pixel times W H / (W H)
    assert abs((power * counts).sum() - (err ** 2).sum(axis=(1, 2)).mean()) < 1e-9
    # cos(2 pi 3 x / W): all power at fx = +-3, fy = 0, each |F|^2 / P = P / 4
    W = H = 32
    x = np.arange(W)
    e = np.tile(np.cos(2 * math.pi * 3 * x / W), (H, 1))[None]
    power, counts = cr.error_spectrum(e)
    total = power * counts
    assert abs(total[3] - W * H / 2) < 1e-9 and abs(total.sum() - W * H / 2) < 1e-9


def test_optimised_tile_has_less_low_frequency_error_power():
    """Fig. 1b: after the optimisation the error's power at low frequencies drops, while the
    total (the per-pixel error multiset is only permuted) stays the same."""
    W = H = 32
    t = oracle.OracleTile(W, H, 16, 64, seed=5)
    p0, c = cr.error_spectrum(cr.heaviside_errors(t.k, t.N, t.a, t.b, t.C, W, H))
    for _ in range(120):
        t.sweep()
    p1, _ = cr.error_spectrum(cr.heaviside_errors(t.k, t.N, t.a, t.b, t.C, W, H))
    low = slice(1, W // 8 + 1)
    assert (p1[low] * c[low]).sum() < 0.5 * (p0[low] * c[low]).sum(), (p0[low], p1[low])
    assert abs((p1 * c).sum() - (p0 * c).sum()) < 1e-12 * (p0 * c).sum()
