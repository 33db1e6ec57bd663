"""Host checks of the tensor-core operand layout helpers (include-only, no GPU): the 128-byte
swizzled K-major offset map, the shared-memory descriptor fields and the kind::f16 instruction
descriptor fields, compiled with nvcc as host code and compared with the layout's rules."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2105_12620_gb300", "csrc")

_SRC = r"""
#include <cstdio>
#include "bn_tcgen05.cuh"
int main() {
    using namespace bn::tc;
    for (unsigned r = 0; r < 128; ++r)
        for (unsigned k = 0; k < 64; ++k) printf("o %u %u %u\n", r, k, sw128_offset(r, k));
    const unsigned long long d = sw128_desc(0x12400u, 3);
    printf("d %llu\n", d);
    printf("i %u\n", idesc_f16_f32(128, 160));
    printf("i %u\n", idesc_f16_f32(128, 16));
    return 0;
}
"""


@pytest.fixture(scope="module")
def values(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("tc")
    src, exe = d / "t.cu", d / "t"
    src.write_text(_SRC)
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    offs, ids, desc = {}, [], None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "o":
            offs[(int(f[1]), int(f[2]))] = int(f[3])
        elif f[0] == "d":
            desc = int(f[1])
        else:
            ids.append(int(f[1]))
    return offs, desc, ids


def test_swizzled_offsets_are_a_permutation_of_the_tile(values):
    offs = values[0]
    seen = sorted(offs.values())
    assert seen == list(range(0, 128 * 128, 2))  # every f16 slot of 128 rows x 128 bytes once


def test_swizzle_rule(values):
    offs = values[0]
    for (r, k), o in offs.items():
        atom, within = divmod(o, 1024)
        assert atom == r // 8                       # 8-row groups 1024 bytes apart
        assert within // 128 == r % 8               # rows 128 bytes apart inside a group
        assert (within % 128) // 16 == (k // 8) ^ (r % 8)   # 16-byte piece XOR row
        assert (within % 16) // 2 == k % 8


def test_eight_rows_of_one_piece_touch_distinct_bank_groups(values):
    offs = values[0]
    for k in range(0, 64, 8):
        groups = {(offs[(r, k)] % 128) // 16 for r in range(8)}
        assert len(groups) == 8


def test_shared_memory_descriptor_fields(values):
    d = values[1]
    start = 0x12400 + 3 * 32
    assert d & 0x3FFF == (start >> 4) & 0x3FFF      # start address >> 4
    assert (d >> 16) & 0x3FFF == 1                  # leading offset (unused by this layout)
    assert (d >> 32) & 0x3FFF == 1024 >> 4          # 8-row groups 1024 bytes apart
    assert (d >> 46) & 0x7 == 1                     # descriptor version
    assert (d >> 49) & 0x7 == 0                     # base offset: atoms 1024-byte aligned
    assert (d >> 61) & 0x7 == 2                     # 128-byte swizzle


def test_instruction_descriptor_fields(values):
    for idesc, n in zip(values[2], (160, 16)):
        assert (idesc >> 4) & 0x3 == 1              # f32 accumulators
        assert (idesc >> 7) & 0x7 == 0 and (idesc >> 10) & 0x7 == 0   # f16 A and B
        assert (idesc >> 13) & 0x3 == 0             # no negation
        assert (idesc >> 15) & 0x3 == 0             # both K-major
        assert (idesc >> 17) & 0x3F == n >> 3
        assert (idesc >> 24) & 0x1F == 128 >> 4
        assert idesc & 0x7 == 0                     # dense
