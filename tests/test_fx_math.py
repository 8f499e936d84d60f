"""Host checks of the two-phase engine's compile-time arithmetic: the cos and
sin of 2 pi m / N its register DFTs are built from (exact angle reduction
and Taylor series, csrc/fx_math.h), compiled as plain C++ and compared with
the C library's values in long double."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1508_02766_gb300", "csrc")

PROG = r"""
#include <cmath>
#include <cstdio>
#include "fx_math.h"
int main() {
  const long long Ns[] = {2,3,4,5,6,7,8,9,10,12,14,15,16,18,20,21,24,25,27,28,30,32,35,36,40,
                          280,1080,1600,4096};
  for (long long N : Ns)
    for (long long m = -N; m < 2 * N; ++m) {
      constexpr long double two_pi = 6.283185307179586476925286766559005768L;
      const kde::fxm::CS cs = kde::fxm::cossin_2pi(m, N);
      const long double a = two_pi * (long double)(((m % N) + N) % N) / (long double)N;
      std::printf("%lld %lld %.17e %.17e %.17Le %.17Le\n", N, m, cs.c, cs.s, cosl(a), sinl(a));
    }
  // values used at compile time must be the same constants
  static_assert(kde::fxm::cossin_2pi(0, 7).c == 1.0, "cos 0");
  static_assert(kde::fxm::cossin_2pi(2, 8).s == 1.0, "sin pi/2");
  return 0;
}
"""


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("fxm")
    src = d / "t.cpp"
    src.write_text(PROG)
    exe = d / "t"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return np.array([[float(x) for x in line.split()] for line in out.splitlines()])


def test_twiddles_match_the_c_library(table):
    err = np.max(np.abs(table[:, 2:4] - table[:, 4:6]))
    assert err <= 4.5e-16, err   # two ulp of the double sums (the kernels use them as floats)


def test_twiddles_have_the_symmetries_of_the_circle(table):
    c, s = table[:, 2], table[:, 3]
    assert np.max(np.abs(c * c + s * s - 1.0)) < 5e-16
    N, m = table[:, 0].astype(np.int64), table[:, 1].astype(np.int64)
    exact = (4 * m) % N == 0          # multiples of a quarter turn are exact
    q = ((4 * m) // N)[exact] % 4
    assert np.array_equal(c[exact], np.array([1.0, 0.0, -1.0, 0.0])[q])
    assert np.array_equal(s[exact], np.array([0.0, 1.0, 0.0, -1.0])[q])
