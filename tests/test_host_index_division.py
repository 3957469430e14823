"""The scatter's 32-bit index decode divides by each axis extent with a
multiply-high and shift (division by invariant integers, Granlund and
Montgomery 1994).  The host routine that derives the multiplier and shift is
compiled here against the library header and checked against exact integer
division: every extent below 70000 on random, boundary and near-multiple
numerators, and random extents up to 2^31."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECK = r'''
#include "kernels.cuh"
#include <cstdio>
#include <random>
static uint32_t umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }
int main() {
  std::mt19937_64 rng(7);
  long bad = 0, n_checks = 0;
  auto chk = [&](uint32_t d, uint32_t n) {
    uint32_t mag; uint8_t shf;
    ttnn::div_magic(d, &mag, &shf);
    const uint32_t q = (uint32_t)(((uint64_t)umulhi(n, mag) + n) >> shf);
    ++n_checks;
    if (q != n / d) ++bad;
  };
  for (uint32_t d = 1; d < 70000; ++d) {
    for (int t = 0; t < 20; ++t) chk(d, (uint32_t)(rng() >> 33));
    for (uint64_t k = 1; k * d < (1ull << 31); k = k * 5 + 1) {
      chk(d, (uint32_t)(k * d));
      chk(d, (uint32_t)(k * d - 1));
    }
    chk(d, 0u);
    chk(d, 0x7fffffffu);
  }
  for (int t = 0; t < 200000; ++t) {
    const uint32_t d = (uint32_t)(rng() % 0x7fffffffu) + 1;
    chk(d, (uint32_t)(rng() >> 33));
    chk(d, (uint32_t)((rng() >> 33) / d * d));
  }
  printf("%ld %ld\n", n_checks, bad);
  return bad != 0;
}
'''


def test_div_magic_matches_integer_division(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    src = tmp_path / "check.cpp"
    src.write_text(CHECK)
    exe = tmp_path / "check"
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", cuda_inc, "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2412_06111_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    n_checks, bad = map(int, out.stdout.split())
    assert n_checks > 1_000_000 and bad == 0
