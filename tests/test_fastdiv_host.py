"""Host check of the multiply-shift index division used by the kernels
(csrc/fastdiv.h): exact for every divisor 1..4096 over n < 2^20 and for
random n up to 2^31 - 1, plus large divisors (extents up to the cell limit)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1610_01388_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <cstdint>
#include <random>
#include "fastdiv.h"
int main() {
    using blbm::FastDiv;
    std::mt19937_64 rng(12345);
    long bad = 0;
    auto check = [&](uint32_t d, uint32_t n) {
        FastDiv f = FastDiv::make(d);
        if (f.div(n) != n / d) { if (bad < 5) printf("d=%u n=%u got %u\n", d, n, f.div(n)); ++bad; }
    };
    for (uint32_t d = 1; d <= 4096; ++d) {
        FastDiv f = FastDiv::make(d);
        for (uint32_t n = 0; n < (1u << 20); n += (d < 64 ? 1 : 7)) if (f.div(n) != n / d) ++bad;
        for (int k = 0; k < 2000; ++k) check(d, uint32_t(rng() % 0x7fffffffu));
        check(d, 0x7fffffffu - 1); check(d, 0x7fffffffu - 64);
    }
    const uint32_t big[] = {65536, 65537, 131071, 262144, 1000003, 16777215, 16777217,
                            123456789, 1073741823, 1073741824, 2147483583u};
    for (uint32_t d : big)
        for (int k = 0; k < 200000; ++k) check(d, uint32_t(rng() % 0x7fffffffu));
    printf("bad=%ld\n", bad);
    return bad != 0;
}
"""


def test_fastdiv_exact(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "t.cpp"
    src.write_text(PROG)
    exe = tmp_path / "t"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
    assert "bad=0" in r.stdout
