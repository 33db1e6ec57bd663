"""CPU oracle for the screen-space sampler optimizer (test infrastructure only).

A thin numpy wrapper over ``bn_oracle.c`` (plain C, double precision), plus the per-tile state
kept as plain numpy arrays.  Only the tests, the smoke check and the CPU-baseline arm of the
benchmark use this package; the product library never imports it.

Method: Belcour & Heitz, "Lessons Learned and Improvements when Building Screen-Space Samplers
with Blue-Noise Error Distribution" (SIGGRAPH '21 Talks).  Sec. 2 (sampler, Eq. 1 loss, test
integrands), Sec. 3.2 (rank-1 lattice + toroidal shift), Sec. 3.4 (parallel swap optimizer).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bn_oracle.c")
_LIB = os.path.join(_HERE, "libbn_oracle.so")

FLAG_VALID, FLAG_IMPROVING, FLAG_COMMITTED, FLAG_TIE = 1, 2, 4, 8
TIE_REL = 1e-6
# +1: reduce Eq. 1 as printed; -1: raise Eq. 1 (= lower the weighted neighbour correlation of
# the estimates, which yields the blue-noise error of Sec. 3.3).  -1 is the default reading.
OBJECTIVE_LITERAL, OBJECTIVE_BLUE = 1, -1
# commit rule: keep only non-interacting improving couples, or every improving couple
MODE_NONINTERACTING, MODE_CONCURRENT = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no architecture-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_i32, _i64, _u32, _u64, _f64 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                ctypes.c_uint64, ctypes.c_double)


def _declare(L):
    L.bno_philox.argtypes = [_u32p, _u32p, _u32p]
    L.bno_van_der_corput.argtypes = [_u32]
    L.bno_van_der_corput.restype = _f64
    L.bno_korobov_min_dist2.argtypes = [_i32, _i32]
    L.bno_korobov_min_dist2.restype = _i64
    L.bno_pick_g.argtypes = [_i32]
    L.bno_pick_g.restype = _i32
    L.bno_points.argtypes = [_i32, _i32, _f64, _f64, _f64p, _f64p]
    L.bno_shifts.argtypes = [_u64, _i32, _i32, _u32p]
    L.bno_heaviside_bank.argtypes = [_u64, _i32, _i32, _i32p, _i32p, _i64p]
    L.bno_perm_rounds.argtypes = [_i32]
    L.bno_perm_rounds.restype = _i32
    L.bno_permutation.argtypes = [_u64, _i32, _i32, _i32p]
    L.bno_counts.argtypes = [_i32, _i32, _i32, _u32p, _i32, _i32p, _i32p, _i64p, _i32p]
    L.bno_torus_d2.argtypes = [_i32, _i32, _i32, _i32]
    L.bno_torus_d2.restype = _i32
    L.bno_energy.argtypes = [_i32, _i32, _i32, _i32, _i32p, _f64, _i32, ctypes.c_void_p]
    L.bno_energy.restype = _f64
    L.bno_delta_energy.argtypes = [_i32, _i32, _i32, _i32, _i32p, _f64, _i32, _i32, _i32,
                                   ctypes.c_void_p]
    L.bno_delta_energy.restype = _f64
    L.bno_sweep_couples.argtypes = [_u64, _i32, _u32, _i32, _i32, _i32p, _i32p]
    L.bno_priority_key.argtypes = [_u64, _i32, _u32, _i32]
    L.bno_priority_key.restype = _u64
    L.bno_sweep.argtypes = [_i32, _i32, _i32, _i32, _f64, _i32, _i32, _i32, _u64, _i32, _u32,
                            _i32, _i32,
                            _i32p, _i32p, _i32p, ctypes.c_void_p, _f64, _f64p, _f64p,
                            _u8p, _i32p]
    L.bno_sweep.restype = _i32


# ---------------------------------------------------------------------------------------------
# function-level wrappers
# ---------------------------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().bno_philox(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def van_der_corput(k: int) -> float:
    return lib().bno_van_der_corput(k)


def korobov_min_dist2(N: int, g: int) -> int:
    return lib().bno_korobov_min_dist2(N, g)


def pick_g(N: int) -> int:
    return lib().bno_pick_g(N)


def points(N: int, g: int, ux: float, uy: float):
    x = np.zeros(N, np.float64)
    y = np.zeros(N, np.float64)
    lib().bno_points(N, g, ux, uy, x, y)
    return x, y


def shifts(seed: int, pair: int, P: int) -> np.ndarray:
    U = np.zeros((P, 2), np.uint32)
    lib().bno_shifts(seed, pair, P, U)
    return U


def heaviside_bank(seed: int, pair: int, T: int):
    a = np.zeros(T, np.int32)
    b = np.zeros(T, np.int32)
    C = np.zeros(T, np.int64)
    lib().bno_heaviside_bank(seed, pair, T, a, b, C)
    return a, b, C


def permutation(seed: int, pair: int, L: int) -> np.ndarray:
    perm = np.zeros(1 << L, np.int32)
    lib().bno_permutation(seed, pair, L, perm)
    return perm


def counts(N: int, g: int, U: np.ndarray, a, b, C) -> np.ndarray:
    U = np.ascontiguousarray(U, np.uint32)
    a = np.ascontiguousarray(a, np.int32)
    b = np.ascontiguousarray(b, np.int32)
    C = np.ascontiguousarray(C, np.int64)
    P, T = U.shape[0], a.shape[0]
    k = np.zeros((P, T), np.int32)
    lib().bno_counts(N, g, P, U, T, a, b, C, k)
    return k


def _counts_part(args):
    return counts(*args)


def counts_parallel(N: int, g: int, U: np.ndarray, a, b, C, workers: int) -> np.ndarray:
    """counts() over pixel ranges in a pool of spawned processes (same arithmetic per pixel;
    spawned, so that it is safe in a process that already uses a GPU)."""
    import multiprocessing as mp
    P = U.shape[0]
    step = max(1, -(-P // (4 * workers)))
    parts = [(N, g, U[i:i + step], a, b, C) for i in range(0, P, step)]
    with mp.get_context("spawn").Pool(workers) as pool:
        return np.concatenate(pool.map(_counts_part, parts), axis=0)


def torus_d2(W: int, H: int, p: int, q: int) -> int:
    return lib().bno_torus_d2(W, H, p, q)


def energy(W: int, H: int, N: int, k: np.ndarray, sigma: float, r: int):
    """Eq. 1 in FP64; returns (E, exact integer sum of |k_p-k_q|^2 per squared distance)."""
    k = np.ascontiguousarray(k, np.int32)
    cls = np.zeros(r * r + 1, np.int64)
    E = lib().bno_energy(W, H, N, k.shape[1], k, sigma, r, cls.ctypes.data)
    return E, cls


def delta_energy(W: int, H: int, N: int, k: np.ndarray, sigma: float, r: int, a: int, b: int):
    k = np.ascontiguousarray(k, np.int32)
    cls = np.zeros(r * r + 1, np.float64)
    dE = lib().bno_delta_energy(W, H, N, k.shape[1], k, sigma, r, a, b, cls.ctypes.data)
    return dE, cls


def sweep_couples(seed: int, pair: int, sweep: int, L: int, M: int, perm: np.ndarray):
    c = np.zeros((M, 2), np.int32)
    lib().bno_sweep_couples(seed, pair, sweep, L, M, np.ascontiguousarray(perm, np.int32), c)
    return c


def priority_key(seed: int, pair: int, sweep: int, j: int) -> int:
    return lib().bno_priority_key(seed, pair, sweep, j)


# ---------------------------------------------------------------------------------------------
# a whole tile (one pair of dimensions), as plain arrays
# ---------------------------------------------------------------------------------------------
@dataclass
class SweepLog:
    dE: np.ndarray        # float64 [M]
    S: np.ndarray         # float64 [M] sum of |per-distance changes|
    flags: np.ndarray     # uint8 [M]
    couples: np.ndarray   # int32 [M, 2]
    committed: int


def log2_ceil(n: int) -> int:
    L = 0
    while (1 << L) < n:
        L += 1
    return L


class OracleTile:
    """State of one 2-D pair: shifts, estimate counts, shift index, candidate permutation."""

    def __init__(self, width, height, n_points, n_integrands, seed, pair=0, generator_g=0,
                 sigma=2.1, radius=6, couples_per_sweep=0, objective=OBJECTIVE_BLUE,
                 mode=MODE_NONINTERACTING, workers=1):
        self.W, self.H, self.N, self.T = width, height, n_points, n_integrands
        self.P = width * height
        self.L = log2_ceil(self.P)
        self.seed, self.pair = seed, pair
        self.sigma, self.r = sigma, radius
        self.objective = objective
        self.mode = mode
        self.g = generator_g if generator_g else pick_g(n_points)
        self.M = couples_per_sweep if couples_per_sweep else max(1, (1 << self.L) // 8)
        self.U = shifts(seed, pair, self.P)
        self.a, self.b, self.C = heaviside_bank(seed, pair, n_integrands)
        self.perm = permutation(seed, pair, self.L)
        if workers > 1:
            self.k = counts_parallel(self.N, self.g, self.U, self.a, self.b, self.C, workers)
        else:
            self.k = counts(self.N, self.g, self.U, self.a, self.b, self.C)
        self.sidx = np.arange(self.P, dtype=np.int32)
        self.sweep_index = 0

    def energy(self) -> float:
        return energy(self.W, self.H, self.N, self.k, self.sigma, self.r)[0]

    def shifts_float(self) -> np.ndarray:
        """u_p as float32 [H, W, 2] (exact: 24 significant bits)."""
        u = self.U[self.sidx].astype(np.float64) / 4294967296.0
        return u.astype(np.float32).reshape(self.H, self.W, 2)

    def sweep(self, gpu_improving: np.ndarray | None = None, tie_rel: float = TIE_REL) -> SweepLog:
        M = self.M
        dE = np.zeros(M, np.float64)
        S = np.zeros(M, np.float64)
        flags = np.zeros(M, np.uint8)
        couples = np.zeros((M, 2), np.int32)
        ptr = None
        if gpu_improving is not None:
            gi = np.ascontiguousarray(gpu_improving, np.uint8)
            ptr = gi.ctypes.data
        committed = lib().bno_sweep(self.W, self.H, self.N, self.T, self.sigma, self.r,
                                    self.objective, self.mode, self.seed, self.pair,
                                    self.sweep_index,
                                    self.L, M,
                                    self.perm, self.k, self.sidx, ptr, tie_rel, dE, S, flags,
                                    couples)
        self.sweep_index += 1
        return SweepLog(dE, S, flags, couples, committed)


# ---------------------------------------------------------------------------------------------
# renderer-side lookup (Sec. 3.1 padding, Sec. 3.2 sampler): samples for a window of screen
# pixels, tile repeated over the screen, dimensions taken in pairs
# ---------------------------------------------------------------------------------------------
def screen_samples(N: int, g: int, U_pairs, W: int, H: int, x0: int, y0: int, width: int,
                   height: int, first: int, count: int, n_dims: int) -> np.ndarray:
    """float64 [height][width][count][n_dims]: sample k = first + j of screen pixel
    (x0 + i, y0 + r) in dimension d is coordinate d % 2 of mod(s^k + u_p, 1) for the tile of
    dimension pair d // 2, with p the tile pixel (x mod W, y mod H).  U_pairs[i] holds the
    shift now at each pixel of pair i ([P, 2] uint32).  An odd n_dims drops the second
    coordinate of the last pair (it is padding)."""
    out = np.zeros((height, width, count, n_dims), np.float64)
    for r in range(height):
        for i in range(width):
            p = ((y0 + r) % H) * W + ((x0 + i) % W)
            for pair in range((n_dims + 1) // 2):
                U = U_pairs[pair]
                x, y = points(N, g, U[p, 0] / 4294967296.0, U[p, 1] / 4294967296.0)
                for j in range(count):
                    k = first + j
                    out[r, i, j, 2 * pair] = x[k]
                    if 2 * pair + 1 < n_dims:
                        out[r, i, j, 2 * pair + 1] = y[k]
    return out
