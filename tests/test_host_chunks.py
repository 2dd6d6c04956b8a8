"""The host pipeline's record-chunk schedule (csrc/host_chunks.h), checked on
the CPU for every small (P_train, P_test): the chunks cover the records in
order, none is empty, there are at most 8, one boundary falls at P_train
(the covariance and solve run there), and with test records the last chunk
holds one record."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2508_11790_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include "host_chunks.h"
int main() {
    int b[9];
    for (int ptr = 1; ptr <= 40; ++ptr)
        for (int pte = 0; pte <= 20; ++pte) {
            const int n = bs::host_chunk_bounds(ptr, pte, 8, b);
            std::printf("%d %d %d", ptr, pte, n);
            for (int i = 0; i <= n; ++i) std::printf(" %d", b[i]);
            std::printf("\n");
        }
    return 0;
}
"""


def test_host_chunk_schedule(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "chunks.cpp"
    exe = tmp_path / "chunks"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = [list(map(int, line.split())) for line in out if line.strip()]
    assert len(rows) == 40 * 21
    for row in rows:
        ptr, pte, n, bounds = row[0], row[1], row[2], row[3:]
        assert len(bounds) == n + 1
        assert 1 <= n <= 8, row
        assert bounds[0] == 0 and bounds[-1] == ptr + pte, row
        assert all(b1 > b0 for b0, b1 in zip(bounds, bounds[1:])), row   # non-empty, in order
        assert ptr in bounds, row                                         # a boundary at P_train
        if pte > 0:
            assert bounds[-1] - bounds[-2] == 1, row                      # last chunk: one record
            assert sum(1 for b in bounds if b > ptr) == min(pte, 3), row  # test chunks
        else:
            assert bounds[-1] == ptr
        assert sum(1 for b in bounds[1:] if b <= ptr) == min(ptr, 8 - min(pte, 3)), row
