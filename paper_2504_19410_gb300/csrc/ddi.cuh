// The 3-D DDI multiplier of Sec. 5, Example 4, evaluated per element inside
// the middle pass.  A middle-pass thread owns one line along axis 1 at fixed
// axis-0 and axis-2 frequencies, so the axis-0/2 parts of n.mu and m.mu are
// set once per line (DdiLine::init) and each element adds its axis-1 part.
// The formula and the parameter block are described with kDdiParCount.
#pragma once
#include <type_traits>

#include "dw.cuh"
#include "fft_core.cuh"
#include "fsa_consts.h"

namespace fsa {

// Middle-pass multiply modes: the stored spectrum alone; the DDI kernel
// reading (cmul * S * D + cadd); the DDI grid reading's derivative on the
// unpadded grid (cmul * D, no spectrum).
enum : int { kMulSpectrum = 0, kMulDdiKernel = 1, kMulDdiGrid = 2 };

// The multiplier is evaluated in FP32 for FP32 plans and in FP64 for FP64
// plans (native or double-word).
template <typename V> struct DdiReal { using T = double; };
template <> struct DdiReal<float2> { using T = float; };

template <typename Q> struct DdiLine {
  Q an, am, bn, bm;   // axes 0 and 2: n.mu0, m.mu0, n.nu, m.nu
  Q n1, m1, w1, nu1;  // axis 1, along the line
  Q cmul, cadd;

  // k0: the axis-0 index (half spectrum; Nyquist at par[kDdiNyq0]); k2: the
  // axis-2 index of a transform of length M2.
  __device__ __forceinline__ void init(const double* __restrict__ par, int k0, int k2, int M2) {
    const bool y0 = k0 == (int)par[kDdiNyq0];
    const int h2 = M2 / 2;
    const bool y2 = k2 == h2;
    const double mu0 = y0 ? 0.0 : (double)k0 * par[kDdiW + 0];
    const double mu2 = y2 ? 0.0 : (double)(k2 < h2 ? k2 : k2 - M2) * par[kDdiW + 2];
    const double nu0 = y0 ? par[kDdiNu + 0] : 0.0;
    const double nu2 = y2 ? par[kDdiNu + 2] : 0.0;
    an = (Q)(par[kDdiN + 0] * mu0 + par[kDdiN + 2] * mu2);
    am = (Q)(par[kDdiM + 0] * mu0 + par[kDdiM + 2] * mu2);
    bn = (Q)(par[kDdiN + 0] * nu0 + par[kDdiN + 2] * nu2);
    bm = (Q)(par[kDdiM + 0] * nu0 + par[kDdiM + 2] * nu2);
    n1 = (Q)par[kDdiN + 1];
    m1 = (Q)par[kDdiM + 1];
    w1 = (Q)par[kDdiW + 1];
    nu1 = (Q)par[kDdiNu + 1];
    cmul = (Q)par[kDdiCmul];
    cadd = (Q)par[kDdiCadd];
  }

  // D at the axis-1 index k1 of a transform of length M1.
  __device__ __forceinline__ Q D(int k1, int M1) const {
    const int h1 = M1 / 2;
    const bool y1 = k1 == h1;
    const Q x = y1 ? Q(0) : (Q)(k1 < h1 ? k1 : k1 - M1) * w1;
    const Q y = y1 ? nu1 : Q(0);
    return -(an + n1 * x) * (am + m1 * x) - (bn + n1 * y) * (bm + m1 * y);
  }

  // The value that multiplies the element: s is the stored spectrum value
  // (kMulDdiKernel) or unused (kMulDdiGrid).
  template <int MODE, typename R> __device__ __forceinline__ R value(R s, int k1, int M1) const {
    const Q d = D(k1, M1);
    if constexpr (std::is_same<R, dw>::value) {
      const double v = MODE == kMulDdiKernel ? cmul * dw_to_double(s) * d + cadd : cmul * d;
      return dw_from_double(v);
    } else {
      return MODE == kMulDdiKernel ? (R)(cmul * (Q)s * d + cadd) : (R)(cmul * d);
    }
  }
};

// phi[0..1] = v + beta * rho[0..1] (the grid reading's -(m.n) rho term),
// added in the precision of the output array.
template <typename V>
__device__ __forceinline__ void store_pair_axpy(typename Io<V>::T* p, V v, double beta, const typename Io<V>::T* r) {
  using T = typename Io<V>::T;
  if constexpr (std::is_same<V, cdw>::value) {
    const double2 a = *reinterpret_cast<const double2*>(r);
    *reinterpret_cast<double2*>(p) = make_double2(dw_to_double(v.x) + beta * a.x, dw_to_double(v.y) + beta * a.y);
  } else {
    const V a = *reinterpret_cast<const V*>(r);
    *reinterpret_cast<V*>(p) = mk(v.x + (T)beta * a.x, v.y + (T)beta * a.y);
  }
}

}  // namespace fsa
