"""The upper tile enumeration of the symmetric-model update (TraceGrid::sym): tile number -> tile (bi, j) of a
square grid of n x n traces with TR traces per tile along i, as the update kernels compute it, checked on
the host against brute force: every tile with bi >= j / TR appears exactly once, in order of rows j, and
the count equals sym_tiles(n, TR).  Compiled from the library's own header with nvcc (host code only)."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2202_04486_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "fft_kernels.cuh"
using namespace smdd;
int main() {
    const int trs[] = {2, 4, 8, 16, 32};
    std::vector<int> ns;
    for (int n = 1; n <= 100; ++n) ns.push_back(n);
    for (int n : {127, 128, 129, 150, 201, 256, 301, 600, 601, 1199, 1200, 1201, 2048}) ns.push_back(n);
    int bad = 0;
    for (int TR : trs)
        for (int n : ns) {
            TraceGrid g;
            g.ni = g.nj = n;
            const int nbi = (n + TR - 1) / TR;
            const long long cnt = sym_tiles(n, TR);
            long long expect = 0;
            for (int j = 0; j < n; ++j) expect += nbi - j / TR;
            if (cnt != expect) { std::printf("count n=%d TR=%d %lld %lld\n", n, TR, cnt, expect); ++bad; continue; }
            std::vector<char> seen((size_t)nbi * n, 0);
            long long prev = -1;
            for (long long b = 0; b < cnt; ++b) {
                const int full = sym_tile_to_full(g, TR, (int)b);
                const int bi = full % nbi, j = full / nbi;
                if (j < 0 || j >= n || bi < j / TR || bi >= nbi || seen[full] || full <= prev) {
                    std::printf("tile n=%d TR=%d bid=%lld -> (%d, %d)\n", n, TR, b, bi, j);
                    ++bad;
                    break;
                }
                seen[full] = 1;
                prev = full;
            }
        }
    std::printf(bad ? "FAIL %d\n" : "OK\n", bad);
    return bad ? 1 : 0;
}
"""


def test_upper_tile_enumeration_is_a_bijection():
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "enum.cu"), os.path.join(d, "enum")
        with open(src, "w") as f:
            f.write(PROGRAM)
        r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC, src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout
