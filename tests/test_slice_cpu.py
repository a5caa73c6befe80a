"""The row slicing of Eq. 2 on the host: make_slice (the same __host__
__device__ function the kernels call) must tile every row exactly -- CTA c's
16-byte groups end where CTA c + 1's begin, the first starts at 0, the last
ends at the row's group count, and each bound equals floor(G * c / P) --
for cluster sizes and for the split two-pass path's CTAs per row (up to 4096),
including group counts where G * P no longer fits in 32 bits."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2609_01864_gb300", "csrc")

PROBE = r"""
#include <cstdio>
#include "credit_rows.cuh"
int main() {
    long long G, P;
    while (std::scanf("%lld %lld", &G, &P) == 2) {
        // a 16-byte aligned FP32 row of exactly G groups (no head, no tail)
        for (int c = 0; c < P; ++c) {
            const credit::RowSlice s = credit::make_slice(0, G * 4, 4, static_cast<int>(P), c);
            std::printf("%lld %lld %lld\n", s.g_lo, s.g_hi,
                        credit::slice_count(s, 4, static_cast<int>(P), c));
        }
    }
    return 0;
}
"""


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    pytest.skip("nvcc not available")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    d = tmp_path_factory.mktemp("slice")
    src = d / "probe.cu"
    src.write_text(PROBE)
    exe = d / "probe"
    subprocess.run([_nvcc(), "-std=c++17", "-O1", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
                    "-gencode", "arch=compute_103a,code=sm_103a", str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    return exe


CASES = [(g, p) for p in (1, 4, 16, 608, 4096) for g in (0, 1, 5, 1 << 20, (1 << 20) + 3, 1048583, 1 << 23,
                                                            (1 << 23) - 1, 6000000)]


def test_make_slice_tiles_every_row_exactly(probe):
    stdin = "".join(f"{g} {p}\n" for g, p in CASES)
    out = subprocess.run([str(probe)], input=stdin, capture_output=True, text=True, check=True).stdout.split("\n")
    k = 0
    for G, P in CASES:
        prev_hi = 0
        total = 0
        for c in range(P):
            lo, hi, cnt = (int(t) for t in out[k].split())
            k += 1
            assert lo == G * c // P and hi == G * (c + 1) // P, (G, P, c, lo, hi)
            assert lo == prev_hi
            assert cnt == (hi - lo) * 4
            prev_hi = hi
            total += cnt
        assert prev_hi == G and total == 4 * G
