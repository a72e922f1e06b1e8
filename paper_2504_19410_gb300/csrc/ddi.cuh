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

// A line's coefficients (see DdiPar): (c0, c1, cN) from the plan's table,
// c2 and cadd global.  An element costs two multiply-adds in the path's own
// arithmetic (FP32; FP64; double-word for double-word plans) and the line
// three loads, issued at the tile's start.
template <typename V> struct DdiCoef { using T = typename RealOf<V>::T; };
template <typename C> struct DdiTriple { C c0, c1, cN; };

// Parameter i of the block in the arithmetic C.
template <typename C> __device__ __forceinline__ C ddi_par(const DdiPar* __restrict__ p, int i);
template <> __device__ __forceinline__ float ddi_par<float>(const DdiPar* __restrict__ p, int i) { return p->f[i]; }
template <> __device__ __forceinline__ double ddi_par<double>(const DdiPar* __restrict__ p, int i) { return p->d[i]; }
template <> __device__ __forceinline__ dw ddi_par<dw>(const DdiPar* __restrict__ p, int i) { return dw(p->f[i], p->lo[i]); }

template <typename V> struct DdiLine {
  using C = typename DdiCoef<V>::T;
  C c0, c1, c2, cN, cadd;

  // k0: the axis-0 index (half spectrum); k2: the axis-2 index of a
  // transform of length M2.
  __device__ __forceinline__ void init(const DdiPar* __restrict__ par, int k0, int k2, int M2) {
    const DdiTriple<C>* row = static_cast<const DdiTriple<C>*>(par->tab) + (long long)k0 * M2 + k2;
    c0 = row->c0;
    c1 = row->c1;
    cN = row->cN;
    c2 = ddi_par<C>(par, kDdiC2);
    cadd = ddi_par<C>(par, kDdiCadd);
  }

  // The value that multiplies the element at the axis-1 index k1 of a
  // transform of length M1: s * cmul D + cadd (kMulDdiKernel, s the stored
  // spectrum value) or cmul D (kMulDdiGrid).
  template <int MODE> __device__ __forceinline__ C value(C s, int k1, int M1) const {
    const int h1 = M1 / 2;
    const C q = C(k1 < h1 ? k1 : k1 - M1);
    const C d = k1 == h1 ? cN : c0 + q * (c1 + c2 * q);
    if constexpr (MODE == kMulDdiKernel) return s * d + cadd;
    else return d;
  }
};

// beta of the grid reading's local term in the output array's precision
template <typename T> __device__ __forceinline__ T ddi_beta(const DdiPar* __restrict__ p) { return ddi_par<T>(p, kDdiBeta); }

// phi[0..1] = v + beta * rho[0..1] (the grid reading's -(m.n) rho term),
// added in the precision of the output array.
// The pair of rho values the epilogue adds, as loaded (FP64 arrays for both
// FP64 arithmetics).
template <typename V> struct PairOf { using T = V; };
template <> struct PairOf<cdw> { using T = double2; };

template <typename V>
__device__ __forceinline__ typename PairOf<V>::T load_rho_pair(const typename Io<V>::T* r) {
  return *reinterpret_cast<const typename PairOf<V>::T*>(r);
}

template <typename V>
__device__ __forceinline__ void store_pair_axpy(typename Io<V>::T* p, V v, typename Io<V>::T beta,
                                                typename PairOf<V>::T a) {
  if constexpr (std::is_same<V, cdw>::value) {
    *reinterpret_cast<double2*>(p) = make_double2(dw_to_double(v.x) + beta * a.x, dw_to_double(v.y) + beta * a.y);
  } else {
    *reinterpret_cast<V*>(p) = mk(v.x + beta * a.x, v.y + beta * a.y);
  }
}

}  // namespace fsa
