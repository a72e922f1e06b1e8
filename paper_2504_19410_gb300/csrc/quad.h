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

// E1(x), x > 0, in long double: series (Abramowitz & Stegun 5.1.11) below 1,
// continued fraction (Press et al., Numerical Recipes, expint; modified
// Lentz) above.
inline long double expint_e1(long double x) {
  if (x < 1.0L) {
    long double sum = 0.0L, term = 1.0L;
    for (int k = 1; k < 60; ++k) {
      term *= -x / k;
      sum += term / k;  // (-x)^k / (k k!)
    }
    return -0.577215664901532860606512090082402431L - logl(x) - sum;
  }
  long double b = x + 1.0L, c = 1.0e300L, d = 1.0L / b, h = d;
  for (int i = 1; i < 400; ++i) {
    const long double an = -(long double)i * i;
    b += 2.0L;
    d = 1.0L / (an * d + b);
    c = b + an / c;
    const long double del = c * d;
    h *= del;
    if (fabsl(del - 1.0L) < 1e-19L) break;
  }
  return h * expl(-x);
}

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

namespace fsa {

// Gauss-Kronrod rule G_n / K_{2n+1} on [-1, 1] (Kronrod's extension of the
// n-point Gauss-Legendre rule), computed on the host in long double:
//   1. the n + 1 new nodes are the zeros of the Stieltjes polynomial
//      E_{n+1}, the monic polynomial of degree n + 1 orthogonal to
//      x^j P_n(x), j = 0 .. n, on [-1, 1]: a linear system for its
//      coefficients, whose moments int x^m P_n(x) dx come from a Gauss-
//      Legendre rule exact for their degree;
//   2. those zeros lie one in each gap of the Gauss nodes and of the end
//      points (the interlacing of Legendre-Kronrod nodes), found by bisection;
//   3. the 2n + 1 weights make the rule exact for P_0 .. P_{2n}: a linear
//      system in the Legendre basis.
// x[0 .. 2n] ascending; wk the Kronrod weights; wg the Gauss weights at the
// Gauss nodes and 0 at the new ones.  Returns false if a step fails.
inline long double legendre_p(int n, long double x) {
  long double p0 = 1, p1 = x;
  if (n == 0) return 1;
  for (int k = 1; k < n; ++k) {
    const long double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Gaussian elimination with partial pivoting on an m x m system (row major);
// the solution replaces b.  False if the matrix is singular.
inline bool solve_dense(int m, long double* A, long double* b) {
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (fabsl(A[r * m + c]) > fabsl(A[piv * m + c])) piv = r;
    if (A[piv * m + c] == 0) return false;
    if (piv != c) {
      for (int k = 0; k < m; ++k) {
        const long double t = A[c * m + k];
        A[c * m + k] = A[piv * m + k];
        A[piv * m + k] = t;
      }
      const long double t = b[c];
      b[c] = b[piv];
      b[piv] = t;
    }
    for (int r = c + 1; r < m; ++r) {
      const long double f = A[r * m + c] / A[c * m + c];
      for (int k = c; k < m; ++k) A[r * m + k] -= f * A[c * m + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = m - 1; c >= 0; --c) {
    long double s = b[c];
    for (int k = c + 1; k < m; ++k) s -= A[c * m + k] * b[k];
    b[c] = s / A[c * m + c];
  }
  return true;
}

inline bool gauss_kronrod(int n, long double* x, long double* wk, long double* wg) {
  const int m = n + 1, N = 2 * n + 1;
  long double xg[64], wgg[64];
  if (n < 1 || n > 30) return false;
  gauss_legendre(n, xg, wgg);
  // moments int_{-1}^{1} x^k P_n(x) dx, k <= 2n + 1, by a rule exact to degree 3n + 2
  long double gx[64], gw[64];
  const int ng = (3 * n + 4) / 2 + 1;
  gauss_legendre(ng, gx, gw);
  auto moment = [&](int k) {
    long double s = 0;
    for (int i = 0; i < ng; ++i) s += gw[i] * powl(gx[i], k) * legendre_p(n, gx[i]);
    return s;
  };
  // E(x) = x^m + sum_{i < m} c_i x^i with int E P_n x^j = 0, j < m
  long double A[32 * 32], b[32];
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < m; ++i) A[j * m + i] = moment(i + j);
    b[j] = -moment(m + j);
  }
  if (!solve_dense(m, A, b)) return false;
  auto E = [&](long double t) {
    long double s = 1;
    for (int i = m - 1; i >= 0; --i) s = s * t + b[i];  // Horner: t^m + ... (leading 1)
    return s;
  };
  // one zero of E in each of the n + 1 gaps of {-1, Gauss nodes, 1}
  long double ek[32];
  for (int g = 0; g < m; ++g) {
    long double lo = g == 0 ? -1.0L : xg[g - 1], hi = g == n ? 1.0L : xg[g];
    long double flo = E(lo);
    if (flo == 0 || flo * E(hi) > 0) return false;
    for (int it = 0; it < 200 && hi - lo > 1e-21L; ++it) {
      const long double mid = 0.5L * (lo + hi), fm = E(mid);
      if ((fm < 0) == (flo < 0)) {
        lo = mid;
        flo = fm;
      } else {
        hi = mid;
      }
    }
    ek[g] = 0.5L * (lo + hi);
  }
  // all nodes ascending: ek[0] < xg[0] < ek[1] < ... < xg[n-1] < ek[n]
  for (int i = 0; i < N; ++i) {
    x[i] = (i % 2 == 0) ? ek[i / 2] : xg[i / 2];
    wg[i] = (i % 2 == 0) ? 0.0L : wgg[i / 2];
  }
  // weights: sum_i w_i P_k(x_i) = int P_k = 2 delta_k0, k < N
  long double B[64 * 64], rhs[64];
  if (N > 64) return false;
  for (int k = 0; k < N; ++k) {
    for (int i = 0; i < N; ++i) B[k * N + i] = legendre_p(k, x[i]);
    rhs[k] = k == 0 ? 2.0L : 0.0L;
  }
  if (!solve_dense(N, B, rhs)) return false;
  for (int i = 0; i < N; ++i) wk[i] = rhs[i];
  return true;
}

}  // namespace fsa
