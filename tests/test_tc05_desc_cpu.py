"""The tcgen05 descriptor encoders (csrc/dm_tc05_desc.h), compiled with g++
on the CPU and checked field by field against the bit tables of the PTX ISA
(the instruction descriptor of kind::f16 and the shared-memory matrix
descriptor), before any GPU run uses them."""
import os
import shutil
import subprocess
import tempfile

import pytest

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1808_10375_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include "dm_tc05_desc.h"
int main() {
  using namespace dmtc;
  printf("%u\n", idesc_f16(kFmtF32, kFmtBF16, kFmtBF16, 128, 256));
  printf("%u\n", idesc_f16(kFmtF16, kFmtF16, kFmtF16, 64, 8, true, false));
  printf("%llu\n", (unsigned long long)smem_desc(0x12400u, 16, 1024, kSw128));
  printf("%llu\n", (unsigned long long)smem_desc(0x3FFF0u + 0x40000u, 2048, 128, kSwNone));
  printf("%u\n", tmem_addr(0x00000020u, 96, 480));
  return 0;
}
"""


def bits(v, lo, hi):
    return (v >> lo) & ((1 << (hi - lo)) - 1)


@pytest.fixture(scope="module")
def values():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "t.cpp"), os.path.join(d, "t")
        open(src, "w").write(PROG)
        subprocess.run([gxx, "-std=c++17", "-I", HDR, src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return [int(x) for x in out]


def test_instruction_descriptor_fields(values):
    d = values[0]   # D F32, A and B BF16, K-major both, M = 128, N = 256
    assert bits(d, 0, 4) == 0                       # dense, no saturation
    assert bits(d, 4, 6) == 1                       # D format F32
    assert bits(d, 6, 7) == 0
    assert bits(d, 7, 10) == 1 and bits(d, 10, 13) == 1   # BF16 operands
    assert bits(d, 13, 15) == 0                     # no negation
    assert bits(d, 15, 16) == 0 and bits(d, 16, 17) == 0  # K-major A and B
    assert bits(d, 17, 23) == 256 // 8
    assert bits(d, 23, 24) == 0
    assert bits(d, 24, 29) == 128 // 16
    assert bits(d, 29, 32) == 0
    e = values[1]   # D F16, F16 operands, A MN-major, M = 64, N = 8
    assert bits(e, 4, 6) == 0 and bits(e, 7, 10) == 0 and bits(e, 15, 16) == 1 and bits(e, 16, 17) == 0
    assert bits(e, 17, 23) == 1 and bits(e, 24, 29) == 4


def test_shared_memory_descriptor_fields(values):
    d = values[2]
    assert bits(d, 0, 14) == 0x12400 >> 4           # start address / 16
    assert bits(d, 14, 16) == 0
    assert bits(d, 16, 30) == 1                     # leading byte offset 16 / 16
    assert bits(d, 32, 46) == 1024 >> 4             # stride byte offset
    assert bits(d, 46, 49) == 0b001                 # fixed value
    assert bits(d, 49, 52) == 0 and bits(d, 52, 53) == 0
    assert bits(d, 53, 61) == 0
    assert bits(d, 61, 64) == 2                     # 128-byte swizzle
    e = values[3]   # addresses wrap to the 18-bit shared window; no swizzle
    assert bits(e, 0, 14) == 0x3FFF0 >> 4
    assert bits(e, 16, 30) == 2048 >> 4 and bits(e, 32, 46) == 128 >> 4 and bits(e, 61, 64) == 0


def test_tensor_memory_address(values):
    assert values[4] == 0x20 + (96 << 16) + 480
