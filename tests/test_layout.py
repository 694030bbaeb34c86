"""The packed layout of the solve operators (csrc/layout.hpp), compiled for
the host: the closed-form row offsets equal the running sums of the row
lengths, and every row starts on a 4-entry (16-byte in float32) boundary,
which the sweeps' bulk copies require."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1604_07378_gb300", "csrc")

CHECK = r"""
#include <cstdio>
#include "layout.hpp"
using namespace hqn;
int main() {
    long long rows = 0;
    for (int nc = 1; nc <= 70; ++nc)
        for (int nr = 0; nr <= 40; nr += 3) {
            const int ldc = pad4(nc), ldr = pad4(nc + nr);
            if (ldc % 4 || ldc < nc || ldc >= nc + 4) { printf("pad4 %d\n", nc); return 1; }
            long long off = 0;
            for (int i = 0; i <= nc + nr; ++i) {
                if (fwd_row_off(i, nc, ldc) != off) { printf("fwd off nc=%d nr=%d i=%d\n", nc, nr, i); return 1; }
                if (off % 4) { printf("fwd align nc=%d i=%d\n", nc, i); return 1; }
                if (i == nc + nr) break;
                const int len = fwd_row_len(i, nc, ldc);
                // a triangle row holds its entries 0..i, a rectangle row all columns
                if (len % 4 || len < (i < nc ? i + 1 : nc) || len > ldc) { printf("fwd len %d %d\n", nc, i); return 1; }
                off += len;
                ++rows;
            }
            off = 0;
            for (int j = 0; j <= nc; ++j) {
                if (bwd_row_off(j, ldr) != off) { printf("bwd off nc=%d nr=%d j=%d\n", nc, nr, j); return 1; }
                if (off % 4) { printf("bwd align nc=%d j=%d\n", nc, j); return 1; }
                if (j == nc) break;
                const int st = bwd_row_start(j);
                // the row keeps its diagonal entry j and everything after it
                if (st % 4 || st > j || j - st > 3) { printf("bwd start %d\n", j); return 1; }
                off += ldr - st;
                ++rows;
            }
        }
    printf("ok %lld\n", rows);
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a C++ compiler")
def test_packed_row_offsets_and_alignment(tmp_path):
    src = tmp_path / "check.cpp"
    src.write_text(CHECK)
    exe = tmp_path / "check"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout
