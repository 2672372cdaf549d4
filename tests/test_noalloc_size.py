"""Scratch limit of the allocation-free solve, checked on the CPU.

dj_sssp_noalloc keeps its scratch in a fixed array inside the library, so it
rejects graphs whose scratch would not fit.  The arithmetic lives in a plain
C++ header; this test compiles a tiny host program against it and checks that
the boundary it computes is exact (the largest accepted pitch fits, the next
one does not) and that the figure include/dj.h and the error message quote is
that boundary on a 152-SM GB300.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2504_03667_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include "dj_noalloc_size.h"
int main() {
  using namespace dj;
  for (int sms : {132, 148, 152, 160}) {
    const int p = noalloc_max_pitch(sms);
    std::printf("%d %d %zu %zu %zu\n", sms, p, noalloc_scratch_bytes(p, sms), noalloc_scratch_bytes(p + 32, sms),
                kNoAllocScratchBytes);
  }
  // small graphs: one CTA per 4-column group, slice of 4 columns
  std::printf("small %zu %d %d\n", noalloc_scratch_bytes(32, 152), noalloc_ctas(32, 152), noalloc_slice_cap(32, 152));
  return 0;
}
"""


@pytest.fixture(scope="module")
def rows(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("noalloc")
    src, exe = d / "size.cpp", d / "size"
    src.write_text(PROG)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    return [ln.split() for ln in out if ln.strip()]


def test_boundary_is_exact(rows):
    for sms, p, need, need_next, cap in (map(int, r) for r in rows if r[0] != "small"):
        assert p % 32 == 0 and p > 100_000
        assert need <= cap < need_next, (sms, p)
        # about 32 bytes per column: two parity copies of 16-byte candidate entries
        assert 30 * p < need < 34 * p


def test_small_graph_scratch(rows):
    small = [r for r in rows if r[0] == "small"][0]
    need, ctas, slice_cap = map(int, small[1:])
    assert ctas == 8 and slice_cap == 4  # pitch 32: eight 4-column groups
    assert need == 256 + 64 + 2 * 8 * 16 + 2 * 8 * 4 * 16


def test_documented_limit_matches(rows):
    p152 = [int(r[1]) for r in rows if r[0] == "152"][0]
    header = open(os.path.join(ROOT, "include", "dj.h")).read()
    quoted = re.search(r"n up to ([0-9,]+) on a\s+\*?\s*152-SM GB300", header)
    assert quoted, "include/dj.h no longer states the 152-SM limit"
    assert int(quoted.group(1).replace(",", "")) == p152
