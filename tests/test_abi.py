"""The C-ABI library loads on any machine and exports every entry point the header declares;
argument validation runs on the host before any device work (no GPU needed)."""
import ctypes
import subprocess

import pytest

from paper_2105_12620_gb300 import _lib as L


@pytest.fixture(scope="module")
def lib():
    from paper_2105_12620_gb300 import build
    build.build()
    return L.load()


def test_header_declares_the_boundary():
    names = L.header_symbols()
    for required in ("bn_sampler_init", "bn_evaluate_energy", "bn_optimize_sweeps",
                     "bn_fetch_shifts", "bn_sampler_destroy", "bn_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in L.header_symbols() if n not in exported]
    assert not missing, missing
    for n in L.header_symbols():
        assert hasattr(lib, n)


def test_binding_covers_the_header():
    assert set(L.header_symbols()) <= set(L._SIGS)


def _cfg(**kw):
    base = dict(width=32, height=32, n_points=16, generator_g=0, n_pairs=1, n_integrands=64,
                sigma=2.1, radius=6, couples_per_sweep=0, mode=0, objective=0, schedule=0, seed=1)
    base.update(kw)
    return L.BnConfig(**base)


@pytest.mark.parametrize("kw,needle", [
    (dict(width=1), "width/height"),
    (dict(height=5000), "width/height"),
    (dict(n_points=12), "power of two"),
    (dict(n_points=2048), "power of two"),
    (dict(generator_g=4), "generator_g"),
    (dict(n_pairs=3), "n_pairs"),
    (dict(n_integrands=0), "n_integrands"),
    (dict(n_integrands=5000), "n_integrands"),
    (dict(n_points=512, n_integrands=512), "2^31"),
    (dict(sigma=0.0), "sigma"),
    (dict(radius=9), "radius"),
    (dict(couples_per_sweep=600), "couples_per_sweep"),
    (dict(mode=7), "mode"),
    (dict(objective=5), "objective"),
    (dict(schedule=9), "schedule"),
])
def test_invalid_configs_are_rejected_on_the_host(lib, kw, needle):
    h = ctypes.c_void_p()
    rc = lib.bn_sampler_init(ctypes.byref(_cfg(**kw)), None, ctypes.byref(h))
    assert rc == L.BN_ERR_INVALID_ARG
    assert needle in lib.bn_last_error().decode()
    assert not h.value


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.bn_sampler_init(None, None, ctypes.byref(h)) == L.BN_ERR_INVALID_ARG
    assert lib.bn_evaluate_energy(None, None) == L.BN_ERR_INVALID_ARG
    assert lib.bn_optimize_sweeps(None, 1, None) == L.BN_ERR_INVALID_ARG
    assert lib.bn_fetch_shifts(None, None, 0, 0) == L.BN_ERR_INVALID_ARG
    lib.bn_sampler_destroy(None)


def test_selftest_arguments_validated_on_the_host(lib):
    assert lib.bn_selftest_wait_timeout(2, 1 << 20) == L.BN_ERR_INVALID_ARG
    assert lib.bn_selftest_wait_timeout(0, 10) == L.BN_ERR_INVALID_ARG


_LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "bn_sampler.h"
#define S(T) printf(#T " size %zu\n", sizeof(T));
#define O(T, F) printf(#T " " #F " %zu\n", offsetof(T, F));
int main(void) {
    S(bn_config) O(bn_config, sigma) O(bn_config, seed)
    S(bn_sweep_stats) S(bn_info) O(bn_info, sweep)
    S(bn_kernel_time) O(bn_kernel_time, launches)
    S(bn_schedule) O(bn_schedule, tsplit)
    S(bn_server_config) O(bn_server_config, tensor_policy) O(bn_server_config, memory_budget_bytes)
    S(bn_request) O(bn_request, n_sweeps) O(bn_request, user_tag)
    S(bn_result) O(bn_result, status) O(bn_result, energy) O(bn_result, t_done)
    S(bn_server_stats) O(bn_server_stats, memory_budget) O(bn_server_stats, tensor_chunks)
    O(bn_server_stats, tunes)
    return 0;
}
"""


def test_ctypes_structs_match_the_c_layout(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", L.os.path.dirname(L.HEADER), str(src), "-o",
                    str(exe)], check=True)
    seen = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True,
                               check=True).stdout.splitlines():
        name, field, value = line.split()
        seen[(name, field)] = int(value)
    py = {"bn_config": L.BnConfig, "bn_sweep_stats": L.BnSweepStats, "bn_info": L.BnInfo,
          "bn_kernel_time": L.BnKernelTime, "bn_schedule": L.BnSchedule,
          "bn_server_config": L.BnServerConfig, "bn_request": L.BnRequest,
          "bn_result": L.BnResult, "bn_server_stats": L.BnServerStats}
    for (name, field), value in seen.items():
        cls = py[name]
        got = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert got == value, (name, field, got, value)


def test_binding_constants_match_the_header(tmp_path):
    """Every #define BN_* value of include/bn_sampler.h equals the binding's constant."""
    import re
    names = re.findall(r"^#define (BN_(?:OK|ERR_\w+|MODE_\w+|OBJECTIVE_\w+|SCHEDULE_\w+|"
                       r"INTEGRANDS_\w+|SERVE_\w+))\b", open(L.HEADER).read(), re.M)
    assert "BN_SCHEDULE_TENSOR" in names
    src = tmp_path / "consts.c"
    src.write_text("#include <stdio.h>\n#include \"bn_sampler.h\"\nint main(void) {\n" +
                   "".join(f'    printf("{n} %d\\n", (int)({n}));\n' for n in names) +
                   "    return 0;\n}\n")
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c99", "-I", L.os.path.dirname(L.HEADER), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.splitlines():
        name, value = line.split()
        assert getattr(L, name) == int(value), name


@pytest.mark.parametrize("kw,needle", [
    (dict(max_slots=0), "max_slots"),
    (dict(max_slots=5000), "max_slots"),
    (dict(sweeps_per_chunk=0), "sweeps_per_chunk"),
    (dict(sweeps_per_chunk=501), "sweeps_per_chunk"),
    (dict(memory_budget_bytes=-1), "budget"),
    (dict(tensor_policy=-1), "tensor_policy"),
    (dict(tensor_policy=3), "tensor_policy"),
])
def test_server_config_validated_on_the_host(lib, kw, needle):
    base = dict(device=0, max_slots=4, sweeps_per_chunk=10, tensor_policy=0,
                memory_budget_bytes=0)
    base.update(kw)
    h = ctypes.c_void_p()
    assert lib.bn_server_create(ctypes.byref(L.BnServerConfig(**base)),
                                ctypes.byref(h)) == L.BN_ERR_INVALID_ARG
    assert needle in lib.bn_last_error().decode()
    assert not h.value


def test_server_null_arguments(lib):
    h = ctypes.c_void_p()
    n = ctypes.c_int32()
    assert lib.bn_server_create(None, ctypes.byref(h)) == L.BN_ERR_INVALID_ARG
    assert lib.bn_server_submit(None, None, None) == L.BN_ERR_INVALID_ARG
    assert lib.bn_server_cancel(None, 1) == L.BN_ERR_INVALID_ARG
    assert lib.bn_server_poll(None, None, 0, ctypes.byref(n)) == L.BN_ERR_INVALID_ARG
    assert lib.bn_server_take_shifts(None, 1, None, 0) == L.BN_ERR_INVALID_ARG
    assert lib.bn_server_get_stats(None, None) == L.BN_ERR_INVALID_ARG
    assert lib.bn_server_drain(None, 0.0) == L.BN_ERR_INVALID_ARG
    lib.bn_server_destroy(None)


def test_criterion_and_lookup_null_arguments(lib):
    assert lib.bn_evaluate_criterion(None, 0, 0, 1, None, 1, None) == L.BN_ERR_INVALID_ARG
    assert lib.bn_export_shift_table(None, 0, None, 0) == L.BN_ERR_INVALID_ARG
    assert lib.bn_generate_samples(None, 0, 0, 1, 1, 0, 1, 1, None, 0, 0) == L.BN_ERR_INVALID_ARG


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """Without the CUDA library there is no fallback: loading raises."""
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        L.load(str(tmp_path / "libbnsampler.so"))
