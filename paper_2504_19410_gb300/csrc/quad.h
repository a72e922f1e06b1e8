// Gauss-Legendre nodes and weights on [-1, 1], computed on the host: the
// roots of the Legendre polynomial P_n by Newton's method from the
// asymptotic first guesses cos(pi (i + 3/4) / (n + 1/2)), P_n and P_n' by the
// three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}; weights
// 2 / ((1 - x^2) P_n'(x)^2).  Used for the kernels whose U^eps or far-field
// bound is a one-dimensional integral without closed form (the Yukawa
// kernels' heat-kernel integrals).
#pragma once
#include <cmath>

namespace fsa {

template <typename F> void gauss_legendre(int n, F* x, F* w) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    long double z = cosl(pi * (i + 0.75L) / (n + 0.5L)), dp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = z;
      for (int k = 1; k < n; ++k) {
        const long double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1);  // P_n'(z)
      const long double dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    long double p0 = 1, p1 = z;
    for (int k = 1; k < n; ++k) {
      const long double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1);
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1);
    const long double wi = 2 / ((1 - z * z) * dp * dp);
    x[i] = (F)(-z);
    x[n - 1 - i] = (F)z;
    w[i] = w[n - 1 - i] = (F)wi;
  }
}

}  // namespace fsa
