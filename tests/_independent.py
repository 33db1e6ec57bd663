"""Independent reference computations used to pin the oracle (test-side only).

Nothing here calls the oracle or the CUDA library: these are closed forms and brute forces
written from the mathematics, so that a mistake in the oracle shows up as a disagreement.
"""
from __future__ import annotations

import math

import numpy as np


def half_plane_area(a: float, b: float, c: float) -> float:
    """Area of {(x, y) in [0,1]^2 : a x + b y < c}: clip the unit square by the half-plane
    (Sutherland-Hodgman) and take the shoelace area of what remains."""
    poly = [(0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (0.0, 1.0)]
    out = []
    f = lambda v: a * v[0] + b * v[1] - c
    for i in range(len(poly)):
        cur, nxt = poly[i], poly[(i + 1) % len(poly)]
        fc, fn = f(cur), f(nxt)
        if fc < 0:
            out.append(cur)
        if (fc < 0) != (fn < 0):
            t = fc / (fc - fn)
            out.append((cur[0] + t * (nxt[0] - cur[0]), cur[1] + t * (nxt[1] - cur[1])))
    if len(out) < 3:
        return 0.0
    area = 0.0
    for i in range(len(out)):
        x0, y0 = out[i]
        x1, y1 = out[(i + 1) % len(out)]
        area += x0 * y1 - x1 * y0
    return abs(area) / 2.0


def torus_d2_bruteforce(W, H, p, q) -> int:
    """Squared distance between pixels p, q on the W x H torus: minimum over all images."""
    px, py = p % W, p // W
    qx, qy = q % W, q // W
    best = None
    for ix in (-1, 0, 1):
        for iy in (-1, 0, 1):
            dx = qx + ix * W - px
            dy = qy + iy * H - py
            d2 = dx * dx + dy * dy
            best = d2 if best is None else min(best, d2)
    return best


def energy_all_pairs(W, H, N, k, sigma, r) -> float:
    """Eq. 1 over every ordered pair of distinct pixels (pure Python, O(P^2 T))."""
    P = W * H
    kk = [list(map(int, row)) for row in np.asarray(k)]
    E = 0.0
    for p in range(P):
        for q in range(P):
            if p == q:
                continue
            d2 = torus_d2_bruteforce(W, H, p, q)
            if d2 > r * r:
                continue
            s = sum((x - y) ** 2 for x, y in zip(kk[p], kk[q]))
            E += math.exp(-d2 / sigma**2) * s / (N * N)
    return E


def stencil_offsets(r):
    """Offsets (dx, dy) != 0 with dx^2 + dy^2 <= r^2 (the neighbourhood on a large tile)."""
    return [(dx, dy) for dy in range(-r, r + 1) for dx in range(-r, r + 1)
            if (dx or dy) and dx * dx + dy * dy <= r * r]


def torus_gaussian_blur(img: np.ndarray, sigma_b: float) -> np.ndarray:
    """Blur a [H, W, ...] tile with a normalised Gaussian of std sigma_b (pixels), wrapping
    around the tile (the tile is repeated over the screen)."""
    H, W = img.shape[:2]
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    # Fourier transform of the periodised Gaussian (sum over aliases is negligible here)
    G = np.exp(-2.0 * (math.pi * sigma_b) ** 2 * (fx * fx + fy * fy))
    F = np.fft.fft2(img, axes=(0, 1))
    shape = G.shape + (1,) * (img.ndim - 2)
    return np.real(np.fft.ifft2(F * G.reshape(shape), axes=(0, 1)))
