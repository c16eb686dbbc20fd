"""The connectivity's division by an invariant divisor (FastDiv in csrc/internal.h: the round-up
multiply of Granlund and Montgomery, PLDI 1994) against plain integer division, compiled from the
library's own header for the host (no GPU): every divisor below 70 000 and a geometric sweep up
to 2^31, each with the dividends 0, 1, d - 1, d, d + 1, 2^31 - 2, 2^31 - 1 and a random one, plus
200 000 random (dividend, divisor) pairs."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1711_02751_gb300", "csrc")

PROGRAM = r"""
#include "internal.h"
#include <cstdint>
#include <cstdio>
int main() {
    using hdgdg::FastDiv;
    unsigned long long bad = 0, checked = 0;
    uint64_t s = 88172645463325252ull;
    auto rnd = [&]() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; };
    auto check = [&](unsigned d, int n) {
        FastDiv f;
        f.set(d);
        ++checked;
        if (f.div(n) != n / (int)d) ++bad;
    };
    for (int pass = 0; pass < 2; ++pass)
        for (unsigned d = 1; d < (pass ? 2147483647u / 2 : 70000u); d = pass ? d * 3 / 2 + 1 : d + 1) {
            const int ns[] = {0, 1, (int)d - 1, (int)d, (int)d + 1, 2147483646, 2147483647, (int)(rnd() & 0x7FFFFFFF)};
            for (int n : ns) check(d, n);
        }
    for (int t = 0; t < 200000; ++t) check((unsigned)(rnd() % 2147483647u) + 1u, (int)(rnd() & 0x7FFFFFFF));
    std::printf("%llu %llu\n", checked, bad);
    return bad != 0;
}
"""


def _cuda_include():
    nvcc = shutil.which("nvcc")
    for root in ([os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))] if nvcc else []) + ["/usr/local/cuda"]:
        inc = os.path.join(root, "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


def test_fastdiv_matches_integer_division(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "fastdiv.cpp"
    exe = tmp_path / "fastdiv"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I" + inc, "-I" + CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=120)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    checked, bad = map(int, r.stdout.split())
    assert r.returncode == 0 and bad == 0 and checked > 500000
