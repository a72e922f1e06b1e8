// Register-resident FFT building blocks (second-generation apply kernels).
//
// A line of length M = R1 * R2 is transformed in two register-resident steps
// (Cooley-Tukey with one shared-memory exchange):
//   step A: for each t < R2, the R1 elements x[t + R2 r] are held by one thread,
//           transformed (length R1), and multiplied by exp(-2 pi i t q / M);
//   step B: for each q < R1, the R2 values of step A with that q are held by one
//           thread and transformed (length R2); they are X[q + R1 s], s < R2.
// The inverse runs the two steps in the opposite order with conjugate factors,
// so a forward transform, a pointwise multiply and an inverse transform need
// only two exchanges, and the multiply happens in registers.
//
// Sub-transforms of length 2, 3, 4, 6, 8, 12, 16, 24 and 32 are fully
// unrolled at compile time (recursive decimation in time); their twiddles are
// compile-time constants cos/sin(2 pi k / 96).
#pragma once
#include <type_traits>

#include "fft_core.cuh"
#include "tw96.h"

namespace fsa {

template <int N> using IC = std::integral_constant<int, N>;

// f(IC<B>), f(IC<B+1>), ..., f(IC<E-1>)
template <int B, int E, class F> __device__ __forceinline__ void sfor(const F& f) {
  if constexpr (B < E) {
    f(IC<B>{});
    sfor<B + 1, E>(f);
  }
}

// a * exp(-+2 pi i E / R) (minus sign forward), E a compile-time integer, R | 96.
template <int R, int E, bool FWD, typename V> __device__ __forceinline__ V twc(V a) {
  using T = typename RealOf<V>::T;
  constexpr int e = ((E % R) + R) % R;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (4 * e == R) {
    return rot_mi<FWD>(a);
  } else if constexpr (2 * e == R) {
    return mk(-a.x, -a.y);
  } else if constexpr (4 * e == 3 * R) {
    return rot_mi<!FWD>(a);
  } else {
    static_assert(96 % R == 0, "sub-transform length must divide 96");
    constexpr int k = e * (96 / R);
    constexpr T c = (T)Tw96::c[k];
    constexpr T s = FWD ? (T)(-Tw96::s[k]) : (T)Tw96::s[k];
    return mk(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

template <int R> constexpr int split_of() {
  return (R % 4 == 0 && R > 4) ? 4 : ((R % 2 == 0 && R > 3) ? 2 : 3);
}

// In-place DFT of x[0..R) in registers, natural order in and out.
template <int R, bool FWD, typename V> __device__ __forceinline__ void rfft(V* x) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2 || R == 3 || R == 4) {
    dft<R, FWD>(x);
  } else {
    constexpr int P = split_of<R>();
    constexpr int Q = R / P;
    V sub[P][Q];
    sfor<0, P>([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      sfor<0, Q>([&](auto mc) {
        constexpr int m = decltype(mc)::value;
        sub[p][m] = x[p + P * m];
      });
      rfft<Q, FWD>(sub[p]);
    });
    sfor<0, Q>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      V t[P];
      sfor<0, P>([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        t[p] = twc<R, p * k, FWD>(sub[p][k]);
      });
      dft<P, FWD>(t);
      sfor<0, P>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        x[k + Q * j] = t[j];
      });
    });
  }
}

// Forward DFT of x[0..R) whose upper half is zero (only x[0..R/2) is read):
// X[2j] = DFT_{R/2}(x)[j], X[2j+1] = DFT_{R/2}(x[r] w_R^r)[j].
template <int R, typename V> __device__ __forceinline__ void rfft_half_in(V* x) {
  static_assert(R % 2 == 0, "even length");
  constexpr int H = R / 2;
  V e[H], o[H];
  sfor<0, H>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    e[r] = x[r];
    o[r] = twc<R, r, true>(x[r]);
  });
  rfft<H, true>(e);
  rfft<H, true>(o);
  sfor<0, H>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    x[2 * j] = e[j];
    x[2 * j + 1] = o[j];
  });
}

// Inverse DFT of a[0..R) of which only the outputs r < R/2 are wanted (left in
// a[0..R/2)): x[r] = IDFT_{R/2}(a_even)[r] + w_R^{-r} IDFT_{R/2}(a_odd)[r].
template <int R, typename V> __device__ __forceinline__ void rifft_half_out(V* a) {
  static_assert(R % 2 == 0, "even length");
  constexpr int H = R / 2;
  V e[H], o[H];
  sfor<0, H>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    e[j] = a[2 * j];
    o[j] = a[2 * j + 1];
  });
  rfft<H, false>(e);
  rfft<H, false>(o);
  sfor<0, H>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    a[r] = cadd(e[r], twc<R, r, false>(o[r]));
  });
}

// Two-factor plan M = R1 * R2 with T = R1 threads per line: step B has one
// sub-transform per thread, step A ceil(R2 / R1).
template <int M_, int R1_, int R2_> struct Plan2 {
  static constexpr int M = M_, R1 = R1_, R2 = R2_, T = R1_;
  static constexpr int PA = (R2_ + R1_ - 1) / R1_;
  static_assert(R1_ * R2_ == M_, "plan factors");
};

template <int M> struct Plan2For;
template <> struct Plan2For<8> { using type = Plan2<8, 2, 4>; };
template <> struct Plan2For<12> { using type = Plan2<12, 3, 4>; };
template <> struct Plan2For<16> { using type = Plan2<16, 4, 4>; };
template <> struct Plan2For<24> { using type = Plan2<24, 3, 8>; };
template <> struct Plan2For<32> { using type = Plan2<32, 4, 8>; };
template <> struct Plan2For<48> { using type = Plan2<48, 4, 12>; };
template <> struct Plan2For<64> { using type = Plan2<64, 8, 8>; };
template <> struct Plan2For<96> { using type = Plan2<96, 8, 12>; };
template <> struct Plan2For<128> { using type = Plan2<128, 8, 16>; };
template <> struct Plan2For<192> { using type = Plan2<192, 12, 16>; };
template <> struct Plan2For<256> { using type = Plan2<256, 16, 16>; };
template <> struct Plan2For<384> { using type = Plan2<384, 16, 24>; };
template <> struct Plan2For<512> { using type = Plan2<512, 16, 32>; };
template <> struct Plan2For<768> { using type = Plan2<768, 24, 32>; };
template <> struct Plan2For<1024> { using type = Plan2<1024, 32, 32>; };

// Step A, forward: thread u handles t = u, u + T, ... < R2.  ld(t, r) returns
// x[t + R2 r]; st(q, t, v) stores the twiddled result for (q, t).
// With HALF (the pruned passes: x[t + R2 r] = 0 for r >= R1/2), only the
// lower half is loaded and the half-input transform is used (R1 even).
template <class P, typename V, bool HALF = false, class Ld, class St>
__device__ __forceinline__ void stepA_fwd(int u, const Ld& ld, const St& st) {
  constexpr int R1 = P::R1, R2 = P::R2;
  constexpr bool H = HALF && (R1 % 2 == 0);
#pragma unroll
  for (int i = 0; i < P::PA; ++i) {
    const int t = u + P::T * i;
    if (P::PA * P::T == R2 || t < R2) {
      V a[R1];
      if constexpr (H) {
#pragma unroll
        for (int r = 0; r < R1 / 2; ++r) a[r] = ld(t, r);
        rfft_half_in<R1>(a);
      } else {
#pragma unroll
        for (int r = 0; r < R1; ++r) a[r] = ld(t, r);
        rfft<R1, true>(a);
      }
#pragma unroll
      for (int q = 1; q < R1; ++q) a[q] = cmul(a[q], twiddle<V, P::M>(t * q));
#pragma unroll
      for (int q = 0; q < R1; ++q) st(q, t, a[q]);
    }
  }
}

// Step A, inverse: ld(q, t) returns the (q, t) value; st(t, r, v) stores x[t + R2 r].
// With HALF (outputs r >= R1/2 are discarded by the crop), only the lower
// half of the outputs is computed and stored (R1 even).
template <class P, typename V, bool HALF = false, class Ld, class St>
__device__ __forceinline__ void stepA_inv(int u, const Ld& ld, const St& st) {
  constexpr int R1 = P::R1, R2 = P::R2;
  constexpr bool H = HALF && (R1 % 2 == 0);
#pragma unroll
  for (int i = 0; i < P::PA; ++i) {
    const int t = u + P::T * i;
    if (P::PA * P::T == R2 || t < R2) {
      V a[R1];
#pragma unroll
      for (int q = 0; q < R1; ++q) a[q] = ld(q, t);
      if constexpr (H) {
        rifft_half_out<R1>(a);
#pragma unroll
        for (int r = 0; r < R1 / 2; ++r) st(t, r, a[r]);
      } else {
        rfft<R1, false>(a);
#pragma unroll
        for (int r = 0; r < R1; ++r) st(t, r, a[r]);
      }
    }
  }
}

// Step B, inverse tail: b[s] (s < R2) of sub-transform q -> inverse length-R2
// transform -> multiplied by exp(+2 pi i t q / M) -> st(q, t, v).
template <class P, typename V, class St>
__device__ __forceinline__ void stepB_inv(int q, V* b, const St& st) {
  rfft<P::R2, false>(b);
#pragma unroll
  for (int t = 0; t < P::R2; ++t) st(q, t, t == 0 ? b[0] : cmulc(b[t], twiddle<V, P::M>(t * q)));
}

}  // namespace fsa
