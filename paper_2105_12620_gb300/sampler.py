"""User-facing wrapper of the C ABI: one ``Sampler`` per tile, ``Batch`` for fused sweeps.

Argument marshalling only; every computation runs in the CUDA library.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib as L


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


@dataclass
class SweepStats:
    sweeps: int
    proposals: int
    improving: int
    committed: int
    ties: int


def _schedule(kind, shape=None, tsplit=0) -> L.BnSchedule:
    bx, by, nt, spw = shape if shape else (0, 0, 0, 0)
    return L.BnSchedule(kind, bx, by, nt, spw, tsplit)


def _unpack(sc: L.BnSchedule) -> dict:
    return {"kind": sc.kind, "shape": (sc.block_x, sc.block_y, sc.threads, sc.slots_per_warp),
            "tsplit": sc.tsplit}


class Sampler:
    """Optimiser state of one tile (n_pairs independent 2-D problems) on the current device."""

    def __init__(self, width: int, height: int, n_points: int, n_integrands: int, seed: int = 0,
                 n_pairs: int = 1, generator_g: int = 0, sigma: float = 2.1, radius: int = 6,
                 couples_per_sweep: int = 0, mode: int = L.BN_MODE_NONINTERACTING,
                 objective: int = L.BN_OBJECTIVE_BLUE, schedule: int = L.BN_SCHEDULE_AUTO,
                 stream=None):
        lib = L.load()
        self.cfg = L.BnConfig(width, height, n_points, generator_g, n_pairs, n_integrands,
                              sigma, radius, couples_per_sweep, mode, objective, schedule, seed)
        self._h = ctypes.c_void_p()
        L.check(lib.bn_sampler_init(ctypes.byref(self.cfg), _stream_handle(stream),
                                    ctypes.byref(self._h)))
        self.width, self.height, self.n_pairs = width, height, n_pairs
        self.n_points, self.n_integrands = n_points, n_integrands
        self.P = width * height
        self.info = self.get_info()

    # -- lifetime ---------------------------------------------------------------------------
    def close(self) -> None:
        if self._h:
            L.load().bn_sampler_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    # -- calls --------------------------------------------------------------------------------
    def get_info(self) -> L.BnInfo:
        info = L.BnInfo()
        L.check(L.load().bn_get_info(self._h, ctypes.byref(info)))
        return info

    def energy(self) -> np.ndarray:
        out = (ctypes.c_double * self.n_pairs)()
        L.check(L.load().bn_evaluate_energy(self._h, out))
        return np.array(out[:], np.float64)

    def energy_into(self, device_ptr: int) -> None:
        L.check(L.load().bn_evaluate_energy_device(self._h, device_ptr))

    def optimize(self, n_sweeps: int, stats: bool = True) -> SweepStats | None:
        st = L.BnSweepStats()
        L.check(L.load().bn_optimize_sweeps(self._h, n_sweeps, ctypes.byref(st) if stats else None))
        if not stats:
            return None
        return SweepStats(st.sweeps, st.proposals, st.improving, st.committed, st.ties)

    def set_schedule(self, kind: int, shape=None, tsplit: int = 0) -> None:
        sc = _schedule(kind, shape, tsplit)
        L.check(L.load().bn_sampler_set_schedule(self._h, ctypes.byref(sc)))

    def set_graph_passes(self, passes: int) -> None:
        """Plain and tensor-core schedules: passes per captured CUDA graph (0 = direct
        launches)."""
        L.check(L.load().bn_sampler_set_graph_passes(self._h, passes))

    def get_schedule(self) -> dict:
        sc = L.BnSchedule()
        L.check(L.load().bn_sampler_get_schedule(self._h, ctypes.byref(sc)))
        return _unpack(sc)

    def autotune(self, trial_sweeps: int = 20) -> dict:
        sc = L.BnSchedule()
        L.check(L.load().bn_sampler_autotune(self._h, trial_sweeps, ctypes.byref(sc)))
        return _unpack(sc)

    def reset(self, seed: int) -> None:
        L.check(L.load().bn_sampler_reset(self._h, seed))

    def set_kernel_timing(self, enable) -> None:
        """True or 1: time the evaluation kernel of every pass; 2: every kernel; 0: none."""
        L.check(L.load().bn_set_kernel_timing(self._h, int(enable)))

    def kernel_times(self) -> dict:
        buf = (L.BnKernelTime * 16)()
        n = ctypes.c_int32()
        L.check(L.load().bn_kernel_times(self._h, buf, 16, ctypes.byref(n)))
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
                for i in range(n.value)}

    def shifts(self) -> np.ndarray:
        out = np.zeros((self.n_pairs, self.height, self.width, 2), np.float32)
        L.check(L.load().bn_fetch_shifts(self._h, out.ctypes.data, out.size, 0))
        return out

    def criterion(self, sigmas, integrands: str = "heaviside", n_integrands: int | None = None,
                  pair: int = 0) -> np.ndarray:
        """Filtered-error RMSE per sigma (Sec. 3.3) for the Heaviside bank or smooth bumps."""
        sig = np.ascontiguousarray(sigmas, np.float32).ravel()
        kind = {"heaviside": L.BN_INTEGRANDS_HEAVISIDE, "gaussian": L.BN_INTEGRANDS_GAUSSIAN}[
            integrands]
        n = n_integrands if n_integrands else (self.n_integrands if kind == 0 else 256)
        out = np.zeros(sig.size, np.float64)
        L.check(L.load().bn_evaluate_criterion(self._h, pair, kind, n, sig.ctypes.data, sig.size,
                                               out.ctypes.data))
        return out

    def spectrum(self, integrands: str = "heaviside", n_integrands: int | None = None,
                 pair: int = 0) -> tuple[np.ndarray, np.ndarray]:
        """Radially averaged power spectrum of the error tiles (Fig. 1b): (power per ring,
        frequencies per ring)."""
        kind = {"heaviside": L.BN_INTEGRANDS_HEAVISIDE, "gaussian": L.BN_INTEGRANDS_GAUSSIAN}[
            integrands]
        n = n_integrands if n_integrands else (self.n_integrands if kind == 0 else 256)
        nr = ctypes.c_int32()
        L.check(L.load().bn_error_spectrum(self._h, pair, kind, n, None, None, 0,
                                           ctypes.byref(nr)))
        power = np.zeros(nr.value, np.float64)
        counts = np.zeros(nr.value, np.int64)
        L.check(L.load().bn_error_spectrum(self._h, pair, kind, n, power.ctypes.data,
                                           counts.ctypes.data, nr.value, ctypes.byref(nr)))
        return power, counts

    def shift_table_into(self, pair: int, device_ptr: int, n_words: int) -> None:
        """Current per-pixel shifts (uint32 [H][W][2]) into device memory, for bn_sample()."""
        L.check(L.load().bn_export_shift_table(self._h, pair, device_ptr, n_words))

    def samples(self, x0: int, y0: int, width: int, height: int, first: int, count: int,
                n_dims: int) -> np.ndarray:
        """Renderer lookup: float32 [height][width][count][n_dims] for a window of the screen."""
        out = np.zeros((height, width, count, n_dims), np.float32)
        L.check(L.load().bn_generate_samples(self._h, x0, y0, width, height, first, count, n_dims,
                                             out.ctypes.data, out.size, 0))
        return out

    def samples_into(self, device_ptr: int, n_floats: int, x0: int, y0: int, width: int,
                     height: int, first: int, count: int, n_dims: int) -> None:
        L.check(L.load().bn_generate_samples(self._h, x0, y0, width, height, first, count, n_dims,
                                             device_ptr, n_floats, 1))

    def shifts_into(self, device_ptr: int, n_floats: int) -> None:
        L.check(L.load().bn_fetch_shifts(self._h, device_ptr, n_floats, 1))

    def points(self, pixel: int, pair: int = 0) -> np.ndarray:
        out = np.zeros((self.n_points, 2), np.float32)
        L.check(L.load().bn_fetch_points(self._h, pair, pixel, out.ctypes.data, out.size))
        return out

    def counts(self, pair: int = 0) -> np.ndarray:
        out = np.zeros((self.P, self.n_integrands), np.int32)
        L.check(L.load().bn_fetch_counts(self._h, pair, out.ctypes.data, out.size))
        return out

    def integrands(self, pair: int = 0):
        T = self.n_integrands
        a = np.zeros(T, np.int32)
        b = np.zeros(T, np.int32)
        C = np.zeros(T, np.int64)
        L.check(L.load().bn_fetch_integrands(self._h, pair, a.ctypes.data, b.ctypes.data,
                                             C.ctypes.data, T))
        return a, b, C

    def permutation(self, pair: int = 0) -> np.ndarray:
        out = np.zeros(1 << self.info.log2_padded, np.int32)
        L.check(L.load().bn_fetch_permutation(self._h, pair, out.ctypes.data, out.size))
        return out

    def sweep_log(self, pair: int = 0):
        M = self.info.couples
        dE = np.zeros(M, np.float32)
        flags = np.zeros(M, np.uint8)
        couples = np.zeros((M, 2), np.int32)
        L.check(L.load().bn_fetch_sweep_log(self._h, pair, dE.ctypes.data, flags.ctypes.data,
                                            couples.ctypes.data, M))
        return dE, flags, couples

    def get_state(self):
        sweep = ctypes.c_int64()
        sidx = np.zeros((self.n_pairs, self.P), np.int32)
        L.check(L.load().bn_get_state(self._h, ctypes.byref(sweep), sidx.ctypes.data, sidx.size))
        return int(sweep.value), sidx

    def set_state(self, sweep: int, shift_index: np.ndarray) -> None:
        sidx = np.ascontiguousarray(shift_index, np.int32)
        L.check(L.load().bn_set_state(self._h, sweep, sidx.ctypes.data, sidx.size))


class Batch:
    """Several samplers whose passes run fused in one launch sequence."""

    def __init__(self, samplers: list[Sampler], stream=None):
        arr = (ctypes.c_void_p * len(samplers))(*[s.handle.value for s in samplers])
        self._h = ctypes.c_void_p()
        self.samplers = list(samplers)
        L.check(L.load().bn_batch_create(arr, len(samplers), _stream_handle(stream),
                                         ctypes.byref(self._h)))

    def optimize(self, n_sweeps: int, stats: bool = True) -> SweepStats | None:
        st = L.BnSweepStats()
        L.check(L.load().bn_batch_optimize(self._h, n_sweeps, ctypes.byref(st) if stats else None))
        if not stats:
            return None
        return SweepStats(st.sweeps, st.proposals, st.improving, st.committed, st.ties)

    def optimize_each(self, n_sweeps_per_member, stats: bool = True) -> SweepStats | None:
        arr = np.ascontiguousarray(n_sweeps_per_member, np.int32)
        st = L.BnSweepStats()
        L.check(L.load().bn_batch_optimize_each(self._h, arr.ctypes.data,
                                                ctypes.byref(st) if stats else None))
        if not stats:
            return None
        return SweepStats(st.sweeps, st.proposals, st.improving, st.committed, st.ties)

    def set_schedule(self, kind: int, shape=None, tsplit: int = 0) -> None:
        sc = _schedule(kind, shape, tsplit)
        L.check(L.load().bn_batch_set_schedule(self._h, ctypes.byref(sc)))

    def set_graph_passes(self, passes: int) -> None:
        L.check(L.load().bn_batch_set_graph_passes(self._h, passes))

    def get_schedule(self) -> dict:
        sc = L.BnSchedule()
        L.check(L.load().bn_batch_get_schedule(self._h, ctypes.byref(sc)))
        return _unpack(sc)

    def autotune(self, trial_sweeps: int = 20) -> dict:
        sc = L.BnSchedule()
        L.check(L.load().bn_batch_autotune(self._h, trial_sweeps, ctypes.byref(sc)))
        return _unpack(sc)

    def close(self) -> None:
        if self._h:
            L.load().bn_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Result:
    request_id: int
    user_tag: int
    status: int
    n_pairs: int
    width: int
    height: int
    energy: tuple
    t_submit: float
    t_admit: float
    t_done: float


class Server:
    """Continuous-batching server: requests (a tile configuration and a pass budget) are queued,
    admitted under a slot and device-memory budget, swept together in fused chunks by a
    background thread of the library, and retired with their final Eq. 1 and shifts."""

    def __init__(self, max_slots: int = 64, sweeps_per_chunk: int = 50,
                 memory_budget_bytes: int = 0, device: int = 0,
                 tensor_policy: int = L.BN_SERVE_TENSOR_TUNED):
        self.cfg = L.BnServerConfig(device, max_slots, sweeps_per_chunk, tensor_policy,
                                    memory_budget_bytes)
        self._h = ctypes.c_void_p()
        L.check(L.load().bn_server_create(ctypes.byref(self.cfg), ctypes.byref(self._h)))

    def submit(self, width: int, height: int, n_points: int, n_integrands: int, n_sweeps: int,
               seed: int = 0, n_pairs: int = 1, generator_g: int = 0, sigma: float = 2.1,
               radius: int = 6, couples_per_sweep: int = 0,
               mode: int = L.BN_MODE_NONINTERACTING, objective: int = L.BN_OBJECTIVE_BLUE,
               user_tag: int = 0) -> int:
        cfg = L.BnConfig(width, height, n_points, generator_g, n_pairs, n_integrands, sigma,
                         radius, couples_per_sweep, mode, objective, L.BN_SCHEDULE_AUTO, seed)
        req = L.BnRequest(cfg, n_sweeps, 0, user_tag)
        rid = ctypes.c_int64()
        L.check(L.load().bn_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid)))
        return rid.value

    def cancel(self, request_id: int) -> None:
        L.check(L.load().bn_server_cancel(self._h, request_id))

    def poll(self, cap: int = 256) -> list[Result]:
        buf = (L.BnResult * cap)()
        n = ctypes.c_int32()
        L.check(L.load().bn_server_poll(self._h, buf, cap, ctypes.byref(n)))
        return [Result(r.request_id, r.user_tag, r.status, r.n_pairs, r.width, r.height,
                       tuple(r.energy[:r.n_pairs]), r.t_submit, r.t_admit, r.t_done)
                for r in buf[:n.value]]

    def take_shifts(self, result: Result) -> np.ndarray:
        out = np.empty((result.n_pairs, result.height, result.width, 2), np.float32)
        L.check(L.load().bn_server_take_shifts(self._h, result.request_id, out.ctypes.data,
                                               out.size))
        return out

    def stats(self) -> dict:
        st = L.BnServerStats()
        L.check(L.load().bn_server_get_stats(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in L.BnServerStats._fields_}

    def drain(self, timeout_s: float = 600.0) -> None:
        L.check(L.load().bn_server_drain(self._h, timeout_s))

    def close(self) -> None:
        if self._h:
            L.load().bn_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
