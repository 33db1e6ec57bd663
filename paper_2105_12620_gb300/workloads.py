"""Synthetic workloads of the optimiser (tile sizes, N, T, pairs, pass budgets); host logic only.

  c1  32 x 32, N = 16, T = 64, 200 passes                    (the small configuration)
  c2  128 x 128, N = 64, T = 1024, 2000 passes               (int8 counts)
  c3  256 x 256, N = 256, two pairs x T = 512, 4000 passes   (int16 counts, 4-D)
  c4  96 tiles, side in {32, 64, 128, 256}, N in {4, 16, 64}, T in {256, 1024}, 2000 passes,
      drawn from numpy's Philox generator with seed 0
Inputs are synthetic by construction (Philox shifts and Heavisides): no dataset is involved.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Tile:
    width: int
    height: int
    n_points: int
    n_integrands: int
    n_pairs: int
    sweeps: int

    def couples(self) -> int:
        """Couples per pass and pair with the default setting, 2^ceil(log2 P) / 8 (at least 1)."""
        P = self.width * self.height
        return max(1, (1 << (P - 1).bit_length()) // 8)

    def proposals(self) -> int:
        """Couples proposed over the pass budget, all pairs (every couple is valid when P is a
        power of two)."""
        return self.couples() * self.n_pairs * self.sweeps


def c1() -> list[Tile]:
    return [Tile(32, 32, 16, 64, 1, 200)]


def c2(tiles: int = 1) -> list[Tile]:
    return [Tile(128, 128, 64, 1024, 1, 2000)] * tiles


def c3() -> list[Tile]:
    return [Tile(256, 256, 256, 512, 2, 4000)]


def c4(seed: int = 0, n: int = 96) -> list[Tile]:
    rng = np.random.Generator(np.random.Philox(seed))
    sides = rng.choice([32, 64, 128, 256], n)
    ns = rng.choice([4, 16, 64], n)
    ts = rng.choice([256, 1024], n)
    return [Tile(int(s), int(s), int(k), int(t), 1, 2000) for s, k, t in zip(sides, ns, ts)]


WORKLOADS = {"c1": c1, "c2": c2, "c3": c3, "c4": c4}
