"""GPU parity of the evaluation criterion (Sec. 3.3 filtered-error RMSE, Sec. 3.5 smooth bumps)
and of the renderer lookup (Sec. 3.1 / 3.2) against the oracle.

Tolerances (FP64 on both sides; the filtered errors at wide sigma are differences of terms up to
~10^4 times larger, so a few ulps of the terms become ~1e-12 of the result): Heaviside 1e-9
relative; bumps 1e-7 relative (the two sides' exp/erf differ by an ulp, amplified by the same
cancellation).  Lookup: bit-exact (every sample is a multiple of 2^-24)."""
import numpy as np
import pytest

import oracle
from oracle import criterion as cr

pytestmark = pytest.mark.gpu

SIGMAS = [0.0, 0.25, 1.0, 2.5, 7.0, 20.0]
RTOL_H, RTOL_B = 1e-9, 1e-7


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


def _lockstep(s, tiles, n):
    """Advance GPU sampler and oracle tiles together (the oracle follows the GPU only on couples
    inside the tie margin) and check the couples and decisions stay identical."""
    for _ in range(n):
        s.optimize(1, stats=False)
        for i, ref in enumerate(tiles):
            _, flags, couples = s.sweep_log(i)
            lg = ref.sweep(gpu_improving=(flags & 2) != 0)
            assert np.array_equal(couples, lg.couples)
            assert np.array_equal(flags & 7, lg.flags & 7)


def _oracle_rmse(ref, kind, n, sigmas):
    if kind == "heaviside":
        err = cr.heaviside_errors(ref.k[:, :n], ref.N, ref.a[:n], ref.b[:n], ref.C[:n], ref.W,
                                  ref.H)
    else:
        err = cr.bump_errors(ref.N, ref.g, ref.U[ref.sidx], cr.bump_bank(ref.seed, ref.pair, n),
                             ref.W, ref.H)
    return cr.rmse(err, sigmas)


@pytest.mark.parametrize("cfg", [
    # (W, H, N, T, pairs, seed, n_bumps)
    (24, 20, 16, 64, 1, 3, 40),
    (13, 17, 128, 40, 1, 4, 17),      # 16-bit counts, odd sides
    (32, 32, 64, 256, 2, 5, 33),      # two pairs
    (5, 3, 4, 9, 1, 6, 5),            # tiny torus: sigma >> tile
])
def test_criterion_matches_oracle(pkg, cfg):
    W, H, N, T, pairs, seed, nb = cfg
    s = pkg.Sampler(W, H, N, T, seed=seed, n_pairs=pairs)
    for pair in range(pairs):
        ref = oracle.OracleTile(W, H, N, T, seed=seed, pair=pair)
        for kind, n, rtol in (("heaviside", T, RTOL_H), ("heaviside", max(1, T // 3), RTOL_H),
                              ("gaussian", nb, RTOL_B)):
            got = s.criterion(SIGMAS, kind, n, pair)
            want = _oracle_rmse(ref, kind, n, SIGMAS)
            np.testing.assert_allclose(got, want, rtol=rtol, atol=0)
    s.close()


def test_criterion_after_optimisation_in_lockstep(pkg):
    W, H, N, T = 32, 24, 16, 96
    s = pkg.Sampler(W, H, N, T, seed=8)
    ref = oracle.OracleTile(W, H, N, T, seed=8)
    _lockstep(s, [ref], 60)
    for kind, n, rtol in (("heaviside", T, RTOL_H), ("gaussian", 24, RTOL_B)):
        np.testing.assert_allclose(s.criterion(SIGMAS, kind, n), _oracle_rmse(ref, kind, n, SIGMAS),
                                   rtol=rtol, atol=0)
    s.close()


def test_criterion_full_size_configuration(pkg):
    """128 x 128, N = 64, T = 1024: every integrand of the bank and 16 bumps."""
    W = H = 128
    s = pkg.Sampler(W, H, 64, 1024, seed=0)
    ref = oracle.OracleTile(W, H, 64, 1024, seed=0)
    sig = [0.0, 0.5, 2.0, 8.0, 20.0]
    np.testing.assert_allclose(s.criterion(sig, "heaviside"), _oracle_rmse(ref, "heaviside", 1024,
                                                                           sig), rtol=RTOL_H)
    np.testing.assert_allclose(s.criterion(sig, "gaussian", 16), _oracle_rmse(ref, "gaussian", 16,
                                                                              sig), rtol=RTOL_B)
    s.close()


def test_optimisation_lowers_the_filtered_error_on_gpu(pkg):
    """Sec. 3.3 / 3.5 on a 64 x 64 tile: the filtered error of the optimised tile is well below
    that of the initial random tile, for the Heavisides and for bumps the optimiser never saw."""
    s = pkg.Sampler(64, 64, 64, 256, seed=2)
    sig = [1.0, 2.0, 4.0, 8.0]
    h0, b0 = s.criterion(sig, "heaviside"), s.criterion(sig, "gaussian", 128)
    raw0 = s.criterion([0.0], "heaviside")
    s.optimize(600, stats=False)
    h1, b1 = s.criterion(sig, "heaviside"), s.criterion(sig, "gaussian", 128)
    # the gain shrinks as sigma approaches the tile size (the tile repeats over the screen)
    assert np.all(h1 < h0) and np.all(h1[:3] < 0.7 * h0[:3]), (h0, h1)
    assert np.all(b1 < b0) and b1[1] < 0.9 * b0[1], (b0, b1)
    # unfiltered: a swap only moves estimates between pixels
    np.testing.assert_allclose(s.criterion([0.0], "heaviside"), raw0, rtol=1e-12)
    s.close()


def _oracle_spectrum(ref, kind, n):
    if kind == "heaviside":
        err = cr.heaviside_errors(ref.k[:, :n], ref.N, ref.a[:n], ref.b[:n], ref.C[:n], ref.W,
                                  ref.H)
    else:
        err = cr.bump_errors(ref.N, ref.g, ref.U[ref.sidx], cr.bump_bank(ref.seed, ref.pair, n),
                             ref.W, ref.H)
    return cr.error_spectrum(err)


def _spectra_close(got, want, rtol):
    # the direct DFT and numpy's FFT round differently: relative to each ring, with a floor of
    # 1e-12 of the largest ring for rings that hold almost no power
    (pg, cg), (pw, cw) = got, want
    assert np.array_equal(cg, cw)
    np.testing.assert_allclose(pg, pw, rtol=rtol, atol=1e-12 * pw.max())


@pytest.mark.parametrize("cfg", [
    # (W, H, N, T, pairs, seed, n_bumps)
    (24, 20, 16, 64, 1, 3, 12),
    (13, 17, 128, 40, 1, 4, 9),       # 16-bit counts, odd sides
    (40, 20, 64, 100, 2, 5, 10),      # 2:1 tile (rings of half-way frequencies), two pairs
    (5, 3, 4, 9, 1, 6, 5),            # tiny torus
])
def test_spectrum_matches_oracle(pkg, cfg):
    W, H, N, T, pairs, seed, nb = cfg
    s = pkg.Sampler(W, H, N, T, seed=seed, n_pairs=pairs)
    for pair in range(pairs):
        ref = oracle.OracleTile(W, H, N, T, seed=seed, pair=pair)
        for kind, n, rtol in (("heaviside", T, RTOL_H), ("heaviside", max(1, T // 3), RTOL_H),
                              ("gaussian", nb, RTOL_B)):
            _spectra_close(s.spectrum(kind, n, pair), _oracle_spectrum(ref, kind, n), rtol)
    s.close()


def test_spectrum_full_size_and_low_frequencies_after_optimisation(pkg):
    """128 x 128, N = 64, T = 1024 against the oracle; then Fig. 1b's claim in lockstep: after the
    optimisation the error power in the lowest rings drops, the total stays (a swap permutes the
    per-pixel errors)."""
    W = H = 128
    s = pkg.Sampler(W, H, 64, 1024, seed=0)
    ref = oracle.OracleTile(W, H, 64, 1024, seed=0)
    p0 = s.spectrum("heaviside")
    _spectra_close(p0, _oracle_spectrum(ref, "heaviside", 1024), RTOL_H)
    small = pkg.Sampler(32, 32, 16, 64, seed=9)
    sref = oracle.OracleTile(32, 32, 16, 64, seed=9)
    q0, c = small.spectrum("heaviside")
    _lockstep(small, [sref], 120)
    q1, _ = small.spectrum("heaviside")
    _spectra_close((q1, c), _oracle_spectrum(sref, "heaviside", 64), RTOL_H)
    low = slice(1, 32 // 8 + 1)
    # 0.57 after 80 passes of this tile
    assert (q1[low] * c[low]).sum() < 0.7 * (q0[low] * c[low]).sum(), (q0[low], q1[low])
    assert abs((q1 * c).sum() - (q0 * c).sum()) < 1e-9 * (q0 * c).sum()
    small.close()
    s.close()


def test_spectrum_rejects_bad_arguments(pkg):
    from paper_2105_12620_gb300 import BnError
    s = pkg.Sampler(16, 16, 16, 32, seed=1)
    with pytest.raises(BnError):
        s.spectrum("heaviside", 33)
    with pytest.raises(BnError):
        s.spectrum("gaussian", 5000)
    s.close()
    big = pkg.Sampler(1100, 8, 4, 8, seed=1)
    with pytest.raises(BnError):
        big.spectrum("heaviside")
    big.close()


def test_criterion_rejects_bad_arguments(pkg):
    from paper_2105_12620_gb300 import BnError
    s = pkg.Sampler(16, 16, 16, 32, seed=1)
    for args in (([1.0], "heaviside", 33), ([float("nan")], "heaviside", 8),
                 ([1.0] * 65, "heaviside", 8), ([1.0], "gaussian", 5000)):
        with pytest.raises(BnError):
            s.criterion(*args)
    s.close()


def test_screen_samples_bit_exact(pkg):
    W, H, N, T = 20, 12, 32, 16
    s = pkg.Sampler(W, H, N, T, seed=9, n_pairs=2)
    refs = [oracle.OracleTile(W, H, N, T, seed=9, pair=i) for i in range(2)]
    for x0, y0, w, h, first, count, dims in ((-33, 7, 45, 30, 0, N, 4), (3, -2, 7, 5, 5, 9, 3),
                                             (100, 100, 1, 1, 31, 1, 1)):
        got = s.samples(x0, y0, w, h, first, count, dims)
        want = oracle.screen_samples(N, refs[0].g, [r.U[r.sidx] for r in refs], W, H, x0, y0, w,
                                     h, first, count, dims)
        assert np.array_equal(got.astype(np.float64), want)
    # after optimisation (oracle in lockstep) the lookup follows the moved shifts
    _lockstep(s, refs, 25)
    got = s.samples(-5, -5, 30, 20, 0, N, 4)
    want = oracle.screen_samples(N, refs[0].g, [r.U[r.sidx] for r in refs], W, H, -5, -5, 30, 20,
                                 0, N, 4)
    assert np.array_equal(got.astype(np.float64), want)
    s.close()


def test_shift_table_and_device_lookup(pkg):
    import torch
    W, H, N, T = 16, 8, 64, 8
    s = pkg.Sampler(W, H, N, T, seed=4)
    ref = oracle.OracleTile(W, H, N, T, seed=4)
    _lockstep(s, [ref], 10)
    table = torch.zeros(2 * W * H, dtype=torch.int64, device="cuda")   # room for uint32 pairs
    s.shift_table_into(0, table.data_ptr(), 4 * W * H)
    torch.cuda.synchronize()
    words = table.cpu().numpy().view(np.uint32)[: 2 * W * H].reshape(W * H, 2)
    assert np.array_equal(words, ref.U[ref.sidx])
    dev = torch.zeros((H, W, N, 2), dtype=torch.float32, device="cuda")
    s.samples_into(dev.data_ptr(), dev.numel(), 0, 0, W, H, 0, N, 2)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), s.samples(0, 0, W, H, 0, N, 2))
    with pytest.raises(Exception):
        s.samples(0, 0, 2, 2, 60, 8, 2)     # beyond N
    with pytest.raises(Exception):
        s.samples(0, 0, 2, 2, 0, 8, 3)      # one pair: at most 2 dimensions
    s.close()
