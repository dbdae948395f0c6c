"""The multiply-high division of the CUDA kernels' site geometry.

Site coordinates come from the checkerboard index through FastDiv
(stg_common.cuh): n / d = (mulhi(n, m) + n) >> s with m, s from make_fastdiv
(the round-up method of Granlund and Montgomery), valid for n < 2^31.  The
host branch of FastDiv::div computes the same formula as the device branch
(64-bit product instead of __umulhi).  This test compiles a host program that
includes the header itself and compares FastDiv with the hardware division
for every divisor 1..4096: at n = 0, 1, around every multiple k d +- 1 for
the first and last multiples below 2^31, and at random n < 2^31.  No GPU.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1111_0125_gb300", "csrc")

PROGRAM = r"""
#include <stdio.h>
#include <stdint.h>
#include "stg_common.cuh"

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint32_t next31(void)
{
    state ^= state << 13; state ^= state >> 7; state ^= state << 17;  /* xorshift64 */
    return (uint32_t)(state >> 33);
}

static int check(const stg::FastDiv &f, uint32_t n, long *bad)
{
    if (n >= 0x80000000u) return 0;
    if (f.div(n) != n / f.d) {
        if (*bad < 10) printf("d=%u n=%u got %u want %u\n", f.d, n, f.div(n), n / f.d);
        ++*bad;
    }
    return 1;
}

int main(void)
{
    long bad = 0, tested = 0;
    for (uint32_t d = 1; d <= 4096; ++d) {
        const stg::FastDiv f = stg::make_fastdiv(d);
        const uint32_t kmax = 0x7fffffffu / d;
        for (uint32_t k = 0; k <= kmax; k += (k < 4096 || k + 4096 > kmax) ? 1 : 997) {
            const uint64_t base = (uint64_t)k * d;
            for (int e = -1; e <= 1; ++e) {
                const int64_t n = (int64_t)base + e;
                if (n >= 0) tested += check(f, (uint32_t)n, &bad);
            }
        }
        for (int r = 0; r < 20000; ++r) tested += check(f, next31(), &bad);
        tested += check(f, 0x7fffffffu, &bad);
    }
    printf("tested %ld bad %ld\n", tested, bad);
    return bad != 0;
}
"""


def _nvcc():
    return shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                    if os.path.exists("/usr/local/cuda/bin/nvcc") else None)


def test_fastdiv_matches_division(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "fastdiv_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "fastdiv_check"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
    assert "bad 0" in r.stdout
