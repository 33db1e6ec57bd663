"""ctypes binding of ``include/bn_sampler.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and forwards its arguments;
all work happens in the CUDA library.  A missing or unloadable library raises ImportError-like
RuntimeError: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbnsampler.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "bn_sampler.h")

BN_OK = 0
BN_ERR_INVALID_ARG, BN_ERR_OOM, BN_ERR_CUDA, BN_ERR_TIMEOUT, BN_ERR_BUSY, BN_ERR_BAD_STATE = (
    -1, -2, -3, -4, -5, -6)
BN_MODE_NONINTERACTING, BN_MODE_CONCURRENT = 0, 1
BN_OBJECTIVE_BLUE, BN_OBJECTIVE_LITERAL = -1, 1
BN_SCHEDULE_AUTO, BN_SCHEDULE_PLAIN, BN_SCHEDULE_PERSISTENT, BN_SCHEDULE_TENSOR = 0, 1, 2, 3
BN_INTEGRANDS_HEAVISIDE, BN_INTEGRANDS_GAUSSIAN = 0, 1
BN_SERVE_TENSOR_TUNED, BN_SERVE_TENSOR_ALWAYS, BN_SERVE_TENSOR_NEVER = 0, 1, 2


class BnConfig(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("n_points", ctypes.c_int32), ("generator_g", ctypes.c_int32),
        ("n_pairs", ctypes.c_int32), ("n_integrands", ctypes.c_int32),
        ("sigma", ctypes.c_float), ("radius", ctypes.c_int32),
        ("couples_per_sweep", ctypes.c_int32), ("mode", ctypes.c_int32),
        ("objective", ctypes.c_int32), ("schedule", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


class BnSweepStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("proposals", ctypes.c_int64),
                ("improving", ctypes.c_int64), ("committed", ctypes.c_int64),
                ("ties", ctypes.c_int64)]


class BnInfo(ctypes.Structure):
    _fields_ = [("generator_g", ctypes.c_int32), ("log2_padded", ctypes.c_int32),
                ("couples", ctypes.c_int32), ("count_bytes", ctypes.c_int32),
                ("row_bytes", ctypes.c_int32), ("n_offsets", ctypes.c_int32),
                ("n_classes", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("sweep", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("reset_h2d_bytes", ctypes.c_int64)]


class BnKernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


class BnSchedule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("block_x", ctypes.c_int32),
                ("block_y", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("slots_per_warp", ctypes.c_int32), ("tsplit", ctypes.c_int32)]


class BnServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_slots", ctypes.c_int32),
                ("sweeps_per_chunk", ctypes.c_int32), ("tensor_policy", ctypes.c_int32),
                ("memory_budget_bytes", ctypes.c_int64)]


class BnRequest(ctypes.Structure):
    _fields_ = [("cfg", BnConfig), ("n_sweeps", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("user_tag", ctypes.c_int64)]


class BnResult(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_int64), ("user_tag", ctypes.c_int64),
                ("status", ctypes.c_int32), ("n_pairs", ctypes.c_int32),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("energy", ctypes.c_double * 2), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class BnServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "submitted", "admitted", "completed", "rejected", "cancelled", "failed", "pending",
        "active", "chunks", "proposals", "memory_in_use", "memory_budget", "tensor_chunks",
        "tunes")]


# CTA shapes instantiated for the persistent kernel: (block_x, block_y, threads, pixels/warp)
PERSISTENT_SHAPES = [(8, 8, 256, 4), (16, 8, 512, 4), (8, 16, 512, 4)]


class BnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bn error {code}: {msg}")
        self.code = code


_P = ctypes.c_void_p
_SIGS = {
    "bn_sampler_init": (ctypes.c_int, [ctypes.POINTER(BnConfig), _P, ctypes.POINTER(_P)]),
    "bn_evaluate_energy": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "bn_optimize_sweeps": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(BnSweepStats)]),
    "bn_fetch_shifts": (ctypes.c_int, [_P, _P, ctypes.c_size_t, ctypes.c_int]),
    "bn_sampler_destroy": (None, [_P]),
    "bn_last_error": (ctypes.c_char_p, []),
    "bn_get_info": (ctypes.c_int, [_P, ctypes.POINTER(BnInfo)]),
    "bn_fetch_points": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t]),
    "bn_fetch_counts": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t]),
    "bn_fetch_integrands": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_size_t]),
    "bn_fetch_permutation": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t]),
    "bn_fetch_sweep_log": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_size_t]),
    "bn_get_state": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), _P, ctypes.c_size_t]),
    "bn_set_state": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_size_t]),
    "bn_evaluate_energy_device": (ctypes.c_int, [_P, _P]),
    "bn_launch_counter": (ctypes.c_int64, []),
    "bn_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64]),
    "bn_sampler_reset": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "bn_set_kernel_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "bn_kernel_times": (ctypes.c_int, [_P, ctypes.POINTER(BnKernelTime), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32)]),
    "bn_sampler_set_schedule": (ctypes.c_int, [_P, ctypes.POINTER(BnSchedule)]),
    "bn_sampler_get_schedule": (ctypes.c_int, [_P, ctypes.POINTER(BnSchedule)]),
    "bn_batch_set_schedule": (ctypes.c_int, [_P, ctypes.POINTER(BnSchedule)]),
    "bn_batch_get_schedule": (ctypes.c_int, [_P, ctypes.POINTER(BnSchedule)]),
    "bn_sampler_set_graph_passes": (ctypes.c_int, [_P, ctypes.c_int32]),
    "bn_batch_set_graph_passes": (ctypes.c_int, [_P, ctypes.c_int32]),
    "bn_sampler_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(BnSchedule)]),
    "bn_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(BnSchedule)]),
    "bn_evaluate_energy_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32,
                                                  ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                  ctypes.c_float, ctypes.c_int32, _P, _P]),
    "bn_evaluate_criterion": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             _P, ctypes.c_int32, _P]),
    "bn_error_spectrum": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         _P, _P, ctypes.c_int32, _P]),
    "bn_export_shift_table": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_size_t]),
    "bn_generate_samples": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, _P, ctypes.c_size_t, ctypes.c_int32]),
    "bn_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, _P,
                                       ctypes.POINTER(_P)]),
    "bn_batch_optimize": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(BnSweepStats)]),
    "bn_batch_optimize_each": (ctypes.c_int, [_P, _P, ctypes.POINTER(BnSweepStats)]),
    "bn_batch_destroy": (None, [_P]),
    "bn_server_create": (ctypes.c_int, [ctypes.POINTER(BnServerConfig), ctypes.POINTER(_P)]),
    "bn_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(BnRequest),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "bn_server_cancel": (ctypes.c_int, [_P, ctypes.c_int64]),
    "bn_server_poll": (ctypes.c_int, [_P, ctypes.POINTER(BnResult), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32)]),
    "bn_server_take_shifts": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_size_t]),
    "bn_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(BnServerStats)]),
    "bn_server_drain": (ctypes.c_int, [_P, ctypes.c_double]),
    "bn_server_destroy": (None, [_P]),
}

_lib = None


def header_symbols() -> list[str]:
    """Names of every entry point declared in include/bn_sampler.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|void|const char \*)\s*\*?\s*(bn_\w+)\s*\(",
                                 text, re.M)))


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the CUDA library (build() must have produced it)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run paper_2105_12620_gb300.build"
                           ".build() first (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int) -> None:
    if rc != BN_OK:
        raise BnError(rc, load().bn_last_error().decode())


def __getattr__(name):
    if name.startswith("bn_") and name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)
