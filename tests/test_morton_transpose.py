"""The 8-axis Morton key of the library (`morton_key8` in common.cuh, Sec. II.C:
the top 64 bits of the bit interleave, planes from the most significant, axis 0
first in a plane) computed as one 8 x 8 bit-matrix transpose must equal the
plain bit-by-bit interleave, for every bits-per-axis value 1..22 and for
coordinates with bits at and above that width.  Host-only: the function is
compiled by nvcc into a small CPU program (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include <random>
#include "common.cuh"

static uint64_t interleave(const uint32_t* q, int D, int bp) {
  uint64_t key = 0;
  int n = 0;
  for (int p = bp - 1; p >= 0 && n < 64; --p)
    for (int k = 0; k < D && n < 64; ++k, ++n) key = (key << 1) | (uint64_t)((q[k] >> p) & 1u);
  return key;
}

int main() {
  std::mt19937_64 rng(7);
  long bad = 0, n = 0;
  for (int bp = 1; bp <= 22; ++bp)
    for (int it = 0; it < 20000; ++it) {
      uint32_t q[8];
      for (int k = 0; k < 8; ++k) {
        const uint64_t r = rng();
        switch (it % 4) {
          case 0: q[k] = (uint32_t)r; break;
          case 1: q[k] = (uint32_t)(r & ((1ull << bp) - 1)); break;
          case 2: q[k] = (r & 1) ? 0xffffffffu : 0u; break;
          default: q[k] = (uint32_t)(r & ((2ull << bp) - 1)); break;
        }
      }
      ++n;
      if (interleave(q, 8, bp) != sfc::morton_key8(q, bp)) ++bad;
    }
  printf("%ld %ld\n", n, bad);
  return bad != 0;
}
"""


def test_morton_key8_equals_the_bit_interleave(tmp_path):
    nvcc = os.environ.get("NVCC", "nvcc")
    if shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "morton8.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "morton8"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1712_06326_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    n, bad = map(int, r.stdout.split())
    assert n == 22 * 20000 and bad == 0 and r.returncode == 0
