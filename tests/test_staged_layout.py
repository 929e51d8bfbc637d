"""The staged layout of a prepared table, checked on the host: every range
the kernels copy into shared memory with one bulk copy starts and ends on
16-byte boundaries, and the sections read with wide loads land on the
boundaries those loads need once the header and the range are staged at a
128-byte boundary (MLP and logarithm-hash parameters: 16 bytes, read four
at a time by the lean 2D kernel's MLP instance; keys: 8; 2D cell records:
16).  A small host program built with nvcc evaluates the library's own
layout functions (blob_geom_dev, staged_range) over table sizes, directory
budgets, algorithms and both kinds of axis; no GPU is used."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2112_03229_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "plan.h"
int main() {
  using namespace ss;
  int bad = 0, cases = 0;
  for (int n = 2; n <= 70000; n = n < 80 ? n + 1 : n * 9 / 8) {
    for (int cap : {16, 64, 100, 256, 1000, 4096, 8192}) {
      for (int cells = 0; cells < 2; ++cells) {
        const BlobGeom g = blob_geom_dev(n, cap, cells != 0);
        for (int algo : {BL_BUCKET, BL_BINARY, BL_BALLOT8, BL_BALLOT16, BL_BALLOT32, BL_SPLINE, BL_MLP,
                         BL_LOGHASH}) {
          BlobHdr h{};
          h.n = n; h.nk = n - 1; h.ns = g.ns; h.stride = g.stride; h.algo = algo; h.D = g.D;
          h.off_mlp = g.off_mlp; h.off_dir = g.off_dir; h.off_keys = g.off_keys; h.off_eyt = g.off_eyt;
          h.staged_end = g.staged_end; h.off_cells = cells ? g.off_cells : -1; h.off_full = g.off_full;
          int lo, hi;
          staged_range(h, lo, hi);
          const int at = (int)sizeof(BlobHdr) - lo;   // staged position of blob offset o: o + at
          ++cases;
          bool ok = sizeof(BlobHdr) % 128 == 0 && lo % 16 == 0 && (hi - lo) % 16 == 0 && hi >= lo;
          if (algo == BL_SPLINE || algo == BL_MLP || algo == BL_LOGHASH)
            ok &= lo <= h.off_mlp && (at + h.off_mlp) % 16 == 0;
          if (algo != BL_BINARY || cells) ok &= lo <= h.off_keys && (at + h.off_keys) % 8 == 0;
          if (cells) ok &= lo <= h.off_cells && (at + h.off_cells) % 16 == 0 && h.staged_end <= hi;
          if (!ok) {
            ++bad;
            if (bad <= 10) printf("n=%d cap=%d cells=%d algo=%d lo=%d hi=%d\n", n, cap, cells, algo, lo, hi);
          }
        }
      }
    }
  }
  printf("cases %d bad %d\n", cases, bad);
  return bad != 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_staged_sections_are_aligned(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "layout.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "layout"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-I" + CSRC,
                        "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad 0" in r.stdout and "cases 0" not in r.stdout, r.stdout
