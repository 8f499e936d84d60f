// Compile-time cos and sin of 2 pi m / N for the register DFTs of the
// two-phase FFT engine.  Plain C++ (constexpr, host and device), no CUDA
// headers, so that a host test can check the values against the C library.
//
// Method: exact integer reduction of the angle to [0, pi/4] (quadrant from
// 4m / N, then the complementary angle above pi/4), then the Taylor series
// of sin and cos about 0, summed to 14 terms in double precision (the
// remainder after the x^27 term is below 1e-22 for |x| <= pi/4).
#pragma once

namespace kde {
namespace fxm {

constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  const double x2 = x * x;
  for (int i = 1; i < 14; ++i) {
    term *= -x2 / (double)((2 * i) * (2 * i + 1));
    sum += term;
  }
  return sum;
}

constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  const double x2 = x * x;
  for (int i = 1; i < 14; ++i) {
    term *= -x2 / (double)((2 * i - 1) * (2 * i));
    sum += term;
  }
  return sum;
}

struct CS {
  double c, s;
};

// (cos, sin) of 2 pi m / N for any integer m and N >= 1.
constexpr CS cossin_2pi(long long m, long long N) {
  m %= N;
  if (m < 0) m += N;
  const long long q = (4 * m) / N;          // quadrant 0..3
  const long long r = 4 * m - q * N;        // angle within it: (pi/2) r / N, 0 <= r < N
  double c = 0.0, s = 0.0;
  if (2 * r <= N) {
    const double phi = (kPi / 2.0) * (double)r / (double)N;
    c = taylor_cos(phi);
    s = taylor_sin(phi);
  } else {
    const double phi = (kPi / 2.0) * (double)(N - r) / (double)N;   // pi/2 - angle
    c = taylor_sin(phi);
    s = taylor_cos(phi);
  }
  switch (q) {
    case 0: return CS{c, s};
    case 1: return CS{-s, c};
    case 2: return CS{-c, -s};
    default: return CS{s, -c};
  }
}

}  // namespace fxm
}  // namespace kde
