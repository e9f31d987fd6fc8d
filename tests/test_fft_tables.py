"""Layout of the shared-memory FFTs' pass twiddle tables (host side of mg_fftp.cuh), no GPU: every pass of every
power-of-two transform (2 .. 8192 points) reads exactly the 8192-point table entries its butterflies need, every
table entry is read, and the 3 * 2^a and 5 * 2^a regions neither overlap nor leave their tables.  Compiled with
nvcc as host code."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_15948_gb300", "csrc")

CHECK = r'''
#include <cstdio>
#include <vector>
#include <algorithm>
#include "mg_fftp.cuh"
using namespace mg;
int main() {
  int bad = 0, n = 0;
  std::vector<int> seen(kPtwCount, 0);
  for (int logM = 1; logM <= 13; ++logM) {
    auto chk = [&](int lp, int logr) {
      if (lp == 0) return;   // the first pass has p = 1: no twiddles
      const int p = 1 << lp;
      for (int j = 0; j < logr; ++j)           // row j holds w^(2^j k), w = exp(-2 pi i / (R p))
        for (int k = 0; k < p; ++k) {
          const int e = ptw_base(lp, logr) + j * p + k;
          if (e < 0 || e >= kPtwCount) { ++bad; continue; }
          seen[e] = 1;
          if (ptw_source(e) != (((1 << j) * k) << (13 - lp - logr))) ++bad;
          ++n;
        }
    };
    int lp = 0;
    for (; logM - lp >= 4; lp += 4) chk(lp, 4);
    if (logM - lp > 0) chk(lp, logM - lp);
  }
  int unused = 0;
  for (int e = 0; e < kPtwCount; ++e) unused += !seen[e];
  int bad3 = 0;
  auto regions = [&](int f, int max_a, int count) {
    std::vector<int> own(count, 0);
    for (int a = 1; a <= max_a; ++a)
      for (int lp2 = 0; lp2 < a; lp2 += 4) {
        const int logr = std::min(4, a - lp2), p = f << lp2;
        for (int r = 0; r < logr; ++r)
          for (int k = 0; k < p; ++k) {
            const int e = ptwf_base(f, a, lp2) + r * p + k;
            if (e < 0 || e >= count || own[e]) ++bad3; else own[e] = 1;
          }
        if (logr < 4) break;
      }
  };
  regions(3, kPtw3MaxA, kPtw3Count);
  regions(5, kPtw5MaxA, kPtw5Count);
  if (ptw3_base(7, 4) != ptwf_base(3, 7, 4)) ++bad3;
  printf("%d %d %d %d\n", n, bad, unused, bad3);
  return 0;
}
'''


def test_pass_twiddle_tables_cover_every_pass_exactly(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "check.cu"
    src.write_text(CHECK)
    exe = tmp_path / "check"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)], check=True, capture_output=True,
                   timeout=300)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split()
    n, bad, unused, bad3 = map(int, out)
    assert n > 0 and bad == 0 and unused == 0 and bad3 == 0, out
