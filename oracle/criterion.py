"""CPU oracle of the sampler-evaluation criterion (test infrastructure only).

Sec. 3.3: a screen-space sampler is rated by how much error is left after denoising; the
denoiser is stood in for by Gaussian filters of standard deviation sigma in [0.25, 20] applied to
the tile of Monte-Carlo estimates of the test integrands, and the criterion is the RMSE of the
filtered estimates against the exact integrals, ||(I_N * k_sigma) - I_ref|| (Fig. 1c).
Sec. 3.5: the same criterion on smooth (low-frequency) integrands, a bank of Gaussian bumps,
shows that the optimised sampler also gives blue-noise error for them.

Readings (the paper leaves these open):
  * the filter is the Gaussian exp(-d^2 / (2 sigma^2)) sampled at integer pixel offsets and made
    periodic on the toroidal tile (sum over all wrapped copies), normalised to sum 1, applied
    separably along x and y; sigma <= 0 means no filter;
  * RMSE = sqrt(mean over integrands and pixels of the squared filtered error);
  * Heaviside reference: the exact area of {a x + b y < C / 2^24} within the unit square;
  * smooth integrands: f(x, y) = exp(-((x - cx)^2 + (y - cy)^2) / (2 s^2)) on the unit square
    (not periodic), cx, cy, s drawn from Philox with tag 7: cx = w0 2^-32, cy = w1 2^-32,
    s = 0.05 + 0.45 w2 2^-32; reference integral in closed form with erf.

Fig. 1b shows the Fourier spectrum of the tile of estimates: the error of an optimised tile has
little power at low frequencies.  `error_spectrum` gives its radial average (readings: the power
of integrand t at frequency (u, v) is |F_t(u, v)|^2 / (W H), F_t the 2-D DFT of the error tile, so
white error of variance s^2 has power s^2 everywhere; frequencies are grouped into rings by their
rounded radius in cycles per pixel times min(W, H); the spectrum is the mean over integrands and
over the frequencies of each ring).

Plain numpy in float64; np.fft serves as the library primitive of the periodic convolution and
of the spectrum.  Only the tests use this module.
"""
from __future__ import annotations

import math

import numpy as np

from . import philox, points

TAG_BUMP = 7


# ---------------------------------------------------------------------------------------------
# exact integrals
# ---------------------------------------------------------------------------------------------
def _integral_clamped_linear(alpha: float, beta: float) -> float:
    """Integral over x in [0, 1] of clamp(alpha + beta x, 0, 1), split at the kinks."""
    cuts = [0.0, 1.0]
    if beta != 0.0:
        for level in (0.0, 1.0):
            x = (level - alpha) / beta
            if 0.0 < x < 1.0:
                cuts.append(x)
    cuts.sort()
    total = 0.0
    for x0, x1 in zip(cuts, cuts[1:]):
        if x1 <= x0:
            continue
        # the clamped function is linear on [x0, x1]: its mean is its value at the midpoint
        xm = 0.5 * (x0 + x1)
        total += (x1 - x0) * min(1.0, max(0.0, alpha + beta * xm))
    return total


def heaviside_area(a: int, b: int, C: int) -> float:
    """Area of {(x, y) in [0,1]^2 : a x + b y < C / 2^24} (the exact integral I_ref)."""
    c = C / 16777216.0
    if b == 0:
        # a x < c on [0, 1]
        if a > 0:
            return min(1.0, max(0.0, c / a))
        return min(1.0, max(0.0, 1.0 - c / a))
    # b > 0: y < (c - a x) / b;  b < 0: y > (c - a x) / b
    frac = _integral_clamped_linear(c / b, -a / b)
    return frac if b > 0 else 1.0 - frac


def bump_bank(seed: int, pair: int, n: int) -> np.ndarray:
    """[n, 3] (cx, cy, s) of the smooth test integrands."""
    out = np.zeros((n, 3), np.float64)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for t in range(n):
        w = philox([t, 0, TAG_BUMP, pair], key)
        out[t] = (w[0] / 4294967296.0, w[1] / 4294967296.0, 0.05 + 0.45 * (w[2] / 4294967296.0))
    return out


def bump_integral(cx: float, cy: float, s: float) -> float:
    """Integral of the bump over the unit square (separable: product of two erf differences)."""
    k = s * math.sqrt(math.pi / 2.0)
    r = s * math.sqrt(2.0)
    ix = k * (math.erf((1.0 - cx) / r) + math.erf(cx / r))
    iy = k * (math.erf((1.0 - cy) / r) + math.erf(cy / r))
    return ix * iy


# ---------------------------------------------------------------------------------------------
# error tiles
# ---------------------------------------------------------------------------------------------
def heaviside_errors(k: np.ndarray, N: int, a, b, C, W: int, H: int) -> np.ndarray:
    """[T, H, W] estimate minus reference, k / N - area, for the Heaviside bank."""
    T = k.shape[1]
    ref = np.array([heaviside_area(int(a[t]), int(b[t]), int(C[t])) for t in range(T)])
    est = k.astype(np.float64) / N                      # [P, T]
    return (est - ref[None, :]).T.reshape(T, H, W)


def bump_errors(N: int, g: int, U_tile: np.ndarray, bank: np.ndarray, W: int,
                H: int) -> np.ndarray:
    """[n, H, W] Monte-Carlo estimate (mean over the pixel's N shifted lattice points) minus the
    exact integral, for each bump; U_tile holds the shift now at each pixel ([P, 2] uint32)."""
    n = bank.shape[0]
    P = W * H
    out = np.zeros((n, P), np.float64)
    ref = np.array([bump_integral(*bank[t]) for t in range(n)])
    for p in range(P):
        x, y = points(N, g, U_tile[p, 0] / 4294967296.0, U_tile[p, 1] / 4294967296.0)
        for t in range(n):
            cx, cy, s = bank[t]
            f = np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * s * s))
            out[t, p] = f.mean() - ref[t]
    return out.reshape(n, H, W)


# ---------------------------------------------------------------------------------------------
# the filter and the criterion
# ---------------------------------------------------------------------------------------------
def periodic_gaussian(n: int, sigma: float) -> np.ndarray:
    """Weights w[d], d = 0..n-1 (offset d mod n), of the wrapped sampled Gaussian, sum 1."""
    w = np.zeros(n, np.float64)
    if sigma <= 0.0:
        w[0] = 1.0
        return w
    reach = int(math.ceil(12.0 * sigma)) + n
    for d in range(n):
        total = 0.0
        j = -(reach // n) - 1
        while j * n + d <= reach:
            x = d + j * n
            total += math.exp(-(x * x) / (2.0 * sigma * sigma))
            j += 1
        w[d] = total
    return w / w.sum()


def blur(err: np.ndarray, sigma: float) -> np.ndarray:
    """Periodic separable Gaussian filter of each [H, W] image of err ([T, H, W])."""
    T, H, W = err.shape
    wx = periodic_gaussian(W, sigma)
    wy = periodic_gaussian(H, sigma)
    # circular convolution: out[y, x] = sum_{dy, dx} wy[dy] wx[dx] err[y - dy, x - dx]; the
    # Gaussian is symmetric, so the sign of the offset does not matter
    kern = np.outer(wy, wx)
    F = np.fft.fft2(err, axes=(1, 2)) * np.fft.fft2(kern)[None, :, :]
    return np.real(np.fft.ifft2(F, axes=(1, 2)))


def rmse(err: np.ndarray, sigmas) -> np.ndarray:
    """Criterion per sigma: sqrt(mean of the squared filtered error) over integrands and pixels."""
    return np.array([math.sqrt(float(np.mean(blur(err, s) ** 2))) for s in sigmas])


# ---------------------------------------------------------------------------------------------
# the error spectrum (Fig. 1b)
# ---------------------------------------------------------------------------------------------
def ring_of(fx: int, fy: int, W: int, H: int) -> int:
    """Ring of the signed frequency (fx, fy) of a W x H tile: floor(rho L + 1/2) with
    rho = sqrt((fx / W)^2 + (fy / H)^2) cycles per pixel and L = min(W, H), i.e. the largest b
    with (2b - 1) W H <= 2 L sqrt((fx H)^2 + (fy W)^2); decided exactly in integers."""
    S = (fx * H) ** 2 + (fy * W) ** 2
    m = math.isqrt(4 * min(W, H) ** 2 * S)   # floor(2 L sqrt(S))
    return (m // (W * H) + 1) // 2


def rings(W: int, H: int) -> tuple[np.ndarray, int]:
    """[H, W] ring of every DFT bin in np.fft.fft2 order (index u is the frequency u, or u - W
    above W / 2; likewise v), and the number of rings."""
    ring = np.zeros((H, W), np.int64)
    for v in range(H):
        fy = v if 2 * v <= H else v - H
        for u in range(W):
            fx = u if 2 * u <= W else u - W
            ring[v, u] = ring_of(fx, fy, W, H)
    return ring, int(ring.max()) + 1


def error_spectrum(err: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Radially averaged power spectrum of the error tiles err [T, H, W]: (power per ring, number
    of frequencies per ring); power = mean over t and over the ring of |F_t|^2 / (W H)."""
    T, H, W = err.shape
    ring, n = rings(W, H)
    pw = (np.abs(np.fft.fft2(err, axes=(1, 2))) ** 2).mean(axis=0) / (W * H)
    counts = np.bincount(ring.ravel(), minlength=n)
    sums = np.bincount(ring.ravel(), weights=pw.ravel(), minlength=n)
    return sums / counts, counts
