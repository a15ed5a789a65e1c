"""Host-side sizing logic of the sort (sort_ws.h), checked on the CPU: the
byte-aligned tile key never needs more radix passes than the workspace is
carved for, its key fits 32 bits and orders like the row-major tile id, and
the workspace grows with every size argument.  Compiles a small C++ driver
against the header; no GPU."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2509_25626_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <initializer_list>
#include <vector_types.h>
#include "sort_ws.h"
using namespace gs;
int main() {
    const unsigned sizes[] = {1, 2, 15, 16, 17, 100, 255, 256, 257, 300, 4095, 4096, 4097, 65535};
    int bad = 0;
    for (unsigned tx : sizes)
        for (unsigned ty : sizes) {
            const TileKeyLayout l = tile_key_layout(tx, ty);
            const unsigned long long T = (unsigned long long)tx * ty;
            if (l.passes < 1 || l.passes > kMaxTilePasses || l.passes > tile_passes_bound(T)) {
                std::printf("passes %u x %u: %d > bound %d\n", tx, ty, l.passes, tile_passes_bound(T));
                ++bad;
            }
            // the largest key fits 32 bits and the key orders like ty * tx_count + x
            const unsigned long long kmax = ((unsigned long long)(ty - 1) << l.shift_y) | (tx - 1);
            if (kmax >> 32) { std::printf("key overflow %u x %u\n", tx, ty); ++bad; }
            if (tx > 1 && ((1ull << l.shift_y) < tx)) { std::printf("tx digits too few %u\n", tx); ++bad; }
        }
    for (long long n : {0LL, 1LL, 1000LL, 1LL << 20})
        for (long long m : {0LL, 1LL, 5000LL, 1LL << 22}) {
            const size_t a = carve_sort_ws(nullptr, n, m, 6700, nullptr);
            const size_t b = carve_sort_ws(nullptr, n + 1, m, 6700, nullptr);
            const size_t c = carve_sort_ws(nullptr, n, m + 1, 6700, nullptr);
            const size_t d = carve_sort_ws(nullptr, n, m, 1ull << 20, nullptr);
            if (b < a || c < a || d < a || (a & 255)) { std::printf("carve not monotone %lld %lld\n", n, m); ++bad; }
        }
    std::printf("%s\n", bad ? "FAIL" : "OK");
    return bad ? 1 : 0;
}
"""


def test_sort_layout_and_workspace(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no g++")
    inc = "/usr/local/cuda/include"
    if not os.path.exists(os.path.join(inc, "vector_types.h")):
        pytest.skip("no CUDA headers")
    src = tmp_path / "drv.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "drv"
    subprocess.run([cxx, "-std=c++17", "-O1", f"-I{inc}", f"-I{CSRC}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout
