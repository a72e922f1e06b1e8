// Device FFT building blocks for the FSA apply path (sm_103a).
//
// A transform of length M = 2n (the doubled grid of Sec. 2.2, Eqs.
// DisFourierSeries / rhoTildeK) runs as a Stockham auto-sort FFT: stage s of
// radix R_s reads R_s elements spaced M/R_s apart, multiplies them by the
// stage twiddles, applies a radix-R_s DFT in registers and writes them back
// spaced by the product of the earlier radices; after the last stage the
// data is in natural order.  Stages exchange data through shared memory in
// place: every thread loads and transforms its butterflies, the CTA
// synchronises, then every thread stores.
//
// Twiddles come from a table of exp(-2 pi i k / 3072) (3072 = 3 * 1024 is a
// multiple of every supported length), built on the host in extended
// precision and rounded once; each translation unit holds its own copy in a
// file-scope __device__ array that the host fills once per device.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "dw.cuh"
#include "fsa_consts.h"

namespace fsa {

// ------------------------------------------------------------ complex ----
__device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }

template <typename V> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<cdw> { using T = dw; };

// Element types at the pass boundaries: T = the real type of rho and phi in
// HBM, S = the stored spectrum's element type.  The double-word tier reads and
// writes FP64 arrays and converts at the boundary.
template <typename V> struct Io;
template <> struct Io<float2> { using T = float; using S = float; };
template <> struct Io<double2> { using T = double; using S = double; };
template <> struct Io<cdw> { using T = double; using S = dw; };

// two consecutive reals of rho as one complex value (a + i b)
template <typename V> __device__ __forceinline__ V load_pair(const typename Io<V>::T* p) {
  if constexpr (std::is_same<V, cdw>::value) {
    const double2 d = *reinterpret_cast<const double2*>(p);
    return mk(dw_from_double(d.x), dw_from_double(d.y));
  } else {
    return *reinterpret_cast<const V*>(p);
  }
}
template <typename V> __device__ __forceinline__ void store_pair(typename Io<V>::T* p, V v) {
  if constexpr (std::is_same<V, cdw>::value) {
    *reinterpret_cast<double2*>(p) = make_double2(dw_to_double(v.x), dw_to_double(v.y));
  } else {
    *reinterpret_cast<V*>(p) = v;
  }
}
template <typename V> __device__ __forceinline__ typename RealOf<V>::T load_spec(const typename Io<V>::S* p) {
  if constexpr (std::is_same<V, cdw>::value) {
    const float2 f = __ldg(reinterpret_cast<const float2*>(p));
    return dw(f.x, f.y);
  } else {
    return __ldg(p);
  }
}

// Canonical form of a value leaving a pass for HBM.  The double-word
// operations skip their closing renormalisation, so a low part can grow past
// half an ulp of its high part over many operations; one TwoSum per part at
// each pass boundary bounds that growth to the operations of one pass.
template <typename V> __device__ __forceinline__ V canon(V v) {
  if constexpr (std::is_same<V, cdw>::value) {
    return mk(dw_two_sum(v.x.hi, v.x.lo), dw_two_sum(v.y.hi, v.y.lo));
  } else {
    return v;
  }
}

template <typename V> __device__ __forceinline__ V czero() { return mk(typename RealOf<V>::T(0), typename RealOf<V>::T(0)); }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// double-word complex products: each part is one fused two-term dot product
__device__ __forceinline__ cdw cmul(cdw a, cdw b) {
  return mk(dw_dot2(a.x, b.x, -a.y, b.y), dw_dot2(a.x, b.y, a.y, b.x));
}
__device__ __forceinline__ cdw cmulc(cdw a, cdw b) {
  return mk(dw_dot2(a.x, b.x, a.y, b.y), dw_dot2(a.y, b.x, -a.x, b.y));
}
template <typename V> __device__ __forceinline__ V cscale(V a, typename RealOf<V>::T s) { return mk(a.x * s, a.y * s); }

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// Paired FP32 arithmetic of sm_100 and later: one instruction adds, subtracts
// or scales both parts of a float2 (add/sub/mul.rn.f32x2 on a register pair).
// The FP32 FFT passes issue about a quarter fewer instructions (measured on
// the 256^3 middle pass: 153 M -> 117 M warp instructions); the FP32 pipes do
// the same work, so the time falls by 2-7 % per pass.
__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
template <> __device__ __forceinline__ float2 cscale<float2>(float2 a, float s) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(make_float2(s, s))));
  return f2_unpack(r);
}
#endif
// -i * a for the forward direction, +i * a for the inverse one
template <bool FWD, typename V> __device__ __forceinline__ V rot_mi(V a) {
  return FWD ? mk(a.y, -a.x) : mk(-a.y, a.x);
}

// ------------------------------------------------------------ codelets ----
template <bool FWD, typename V> __device__ __forceinline__ void dft2(V* v) {
  V a = v[0];
  v[0] = cadd(a, v[1]);
  v[1] = csub(a, v[1]);
}

template <bool FWD, typename V> __device__ __forceinline__ void dft3(V* v) {
  using R = typename RealOf<V>::T;
  const R s = R(0.86602540378443864676372317075294);  // sin(2 pi / 3)
  V t1 = cadd(v[1], v[2]);
  V t2 = mk(v[0].x - R(0.5) * t1.x, v[0].y - R(0.5) * t1.y);
  V d = rot_mi<FWD>(cscale(csub(v[1], v[2]), s));
  v[0] = cadd(v[0], t1);
  v[1] = cadd(t2, d);
  v[2] = csub(t2, d);
}

template <bool FWD, typename V> __device__ __forceinline__ void dft4(V* v) {
  V a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  V c = cadd(v[1], v[3]), d = rot_mi<FWD>(csub(v[1], v[3]));
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}

// b_k *= w8^k (k = 1, 2, 3), w8 = exp(-+ 2 pi i / 8)
template <bool FWD, typename V> __device__ __forceinline__ void rot8(V* b) {
  using R = typename RealOf<V>::T;
  const R h = R(0.70710678118654752440084436210485);  // 1/sqrt(2)
  if (FWD) {
    b[1] = mk(h * (b[1].x + b[1].y), h * (b[1].y - b[1].x));
    b[3] = mk(h * (b[3].y - b[3].x), -h * (b[3].x + b[3].y));
  } else {
    b[1] = mk(h * (b[1].x - b[1].y), h * (b[1].x + b[1].y));
    b[3] = mk(-h * (b[3].x + b[3].y), h * (b[3].x - b[3].y));
  }
  b[2] = rot_mi<FWD>(b[2]);
}

template <bool FWD, typename V> __device__ __forceinline__ void dft8(V* v) {
  V a[4], b[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = cadd(v[k], v[k + 4]);
    b[k] = csub(v[k], v[k + 4]);
  }
  rot8<FWD>(b);
  dft4<FWD>(a);
  dft4<FWD>(b);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[2 * q] = a[q];
    v[2 * q + 1] = b[q];
  }
}

// Pruned codelets.  dft_half_in: DFT of v[0..R) whose upper half is zero
// (only v[0..R/2) is read); adding or subtracting the zero half is exact, so
// the results are those of the full codelet.  dft_half_out: only the outputs
// v[0..R/2) are formed.  R in {2, 4, 8}.
template <bool FWD, typename V> __device__ __forceinline__ void dft4_lo2(const V* v, V& o0, V& o1) {
  const V a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  const V c = cadd(v[1], v[3]), d = rot_mi<FWD>(csub(v[1], v[3]));
  o0 = cadd(a, c);
  o1 = cadd(b, d);
}

template <int R, bool FWD, typename V> __device__ __forceinline__ void dft_half_in(V* v) {
  static_assert(R == 2 || R == 4 || R == 8, "pruned codelet radix");
  if constexpr (R == 2) {
    v[1] = v[0];
  } else if constexpr (R == 4) {
    const V a = v[0], c = v[1], d = rot_mi<FWD>(v[1]);
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(a, d);
    v[3] = csub(a, d);
  } else {
    V a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = b[k] = v[k];
    rot8<FWD>(b);
    dft4<FWD>(a);
    dft4<FWD>(b);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[2 * q] = a[q];
      v[2 * q + 1] = b[q];
    }
  }
}

template <int R, bool FWD, typename V> __device__ __forceinline__ void dft_half_out(V* v) {
  static_assert(R == 2 || R == 4 || R == 8, "pruned codelet radix");
  if constexpr (R == 2) {
    v[0] = cadd(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4_lo2<FWD>(v, v[0], v[1]);
  } else {
    V a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] = cadd(v[k], v[k + 4]);
      b[k] = csub(v[k], v[k + 4]);
    }
    rot8<FWD>(b);
    dft4_lo2<FWD>(a, v[0], v[2]);
    dft4_lo2<FWD>(b, v[1], v[3]);
  }
}

template <int R, bool FWD, typename V> __device__ __forceinline__ void dft(V* v) {
  if constexpr (R == 2) dft2<FWD>(v);
  else if constexpr (R == 3) dft3<FWD>(v);
  else if constexpr (R == 4) dft4<FWD>(v);
  else if constexpr (R == 8) dft8<FWD>(v);
  else static_assert(R == 2, "unsupported radix");
}

// ------------------------------------------------------------ plans ------
template <int M_, int... Rs> struct Plan {
  static constexpr int M = M_;
  static constexpr int NST = sizeof...(Rs);
  static constexpr int R[NST] = {Rs...};
  static constexpr int rmax() {
    int m = 1;
    for (int i = 0; i < NST; ++i) m = R[i] > m ? R[i] : m;
    return m;
  }
  static constexpr int ns(int s) {
    int p = 1;
    for (int i = 0; i < s; ++i) p *= R[i];
    return p;
  }
};

// Radix plan per supported length 2n, n in {4,6,8,12,...,384,512}.
template <int M> struct PlanFor;
template <> struct PlanFor<8> { using type = Plan<8, 8>; };
template <> struct PlanFor<12> { using type = Plan<12, 4, 3>; };
template <> struct PlanFor<16> { using type = Plan<16, 4, 4>; };
template <> struct PlanFor<24> { using type = Plan<24, 8, 3>; };
template <> struct PlanFor<32> { using type = Plan<32, 8, 4>; };
template <> struct PlanFor<48> { using type = Plan<48, 4, 4, 3>; };
template <> struct PlanFor<64> { using type = Plan<64, 8, 8>; };
template <> struct PlanFor<96> { using type = Plan<96, 8, 4, 3>; };
template <> struct PlanFor<128> { using type = Plan<128, 8, 4, 4>; };
template <> struct PlanFor<192> { using type = Plan<192, 8, 8, 3>; };
template <> struct PlanFor<256> { using type = Plan<256, 8, 8, 4>; };
template <> struct PlanFor<384> { using type = Plan<384, 8, 4, 4, 3>; };
template <> struct PlanFor<512> { using type = Plan<512, 8, 8, 8>; };
template <> struct PlanFor<768> { using type = Plan<768, 8, 8, 4, 3>; };
template <> struct PlanFor<1024> { using type = Plan<1024, 8, 8, 4, 4>; };

#define FSA_FOR_EACH_M(X) \
  X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)

}  // namespace fsa

// ------------------------------------------------------------ twiddles ---
// One copy per translation unit that includes this header.
static __device__ float2 g_tw32[fsa::kTwN];
static __device__ double2 g_tw64[fsa::kTwN];
static __device__ fsa::cdw g_twdw[fsa::kTwN];

namespace fsa {

template <typename V> __device__ __forceinline__ const V* tw_table();
template <> __device__ __forceinline__ const float2* tw_table<float2>() { return g_tw32; }
template <> __device__ __forceinline__ const double2* tw_table<double2>() { return g_tw64; }
template <> __device__ __forceinline__ const cdw* tw_table<cdw>() { return g_twdw; }

// exp(-2 pi i e / L) for 0 <= e < L, L | 3072
template <typename V, int L> __device__ __forceinline__ V twiddle(int e) {
  static_assert(kTwN % L == 0, "length must divide the twiddle table");
  if constexpr (std::is_same<V, cdw>::value) {
    const float4 f = __ldg(reinterpret_cast<const float4*>(tw_table<V>() + e * (kTwN / L)));
    return mk(dw(f.x, f.y), dw(f.z, f.w));
  } else {
    return __ldg(tw_table<V>() + e * (kTwN / L));
  }
}

// One Stockham stage S of plan P over a line, with T threads per line and
// thread index t.  `ld(p)` returns element p of the stage input, `st(p, v)`
// stores element p of the stage output.  All threads of the CTA must call it
// (it contains two barriers: between loads and stores, and after stores).
// ZIN (first stage, even radix): inputs p >= M/2 are zero, i.e. r >= R/2 --
// they are neither loaded nor transformed.  ZOUT (last stage, even radix):
// only outputs p < M/2, i.e. r < R/2, are formed and stored.
template <class P, int S, bool FWD, int T, typename V, bool ZIN, bool ZOUT, class Ld, class St>
__device__ __forceinline__ void stage(int t, const Ld& ld, const St& st) {
  constexpr int R = P::R[S];
  constexpr int NS = P::ns(S);
  constexpr int M = P::M;
  constexpr int NB = M / R;
  constexpr int PER = (NB + T - 1) / T;
  constexpr bool HIN = ZIN && S == 0 && R % 2 == 0;
  constexpr bool HOUT = ZOUT && S == P::NST - 1 && R % 2 == 0;
  constexpr int RIN = HIN ? R / 2 : R;
  constexpr int ROUT = HOUT ? R / 2 : R;
  V v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = t + q * T;
    if (PER * T == NB || b < NB) {
#pragma unroll
      for (int r = 0; r < RIN; ++r) v[q][r] = ld(b + r * NB);
      if constexpr (NS > 1) {
        const int k = b % NS;
#pragma unroll
        for (int r = 1; r < RIN; ++r) {
          const V w = twiddle<V, NS * R>(r * k);
          v[q][r] = FWD ? cmul(v[q][r], w) : cmulc(v[q][r], w);
        }
      }
      if constexpr (HIN) {
        dft_half_in<R, FWD>(v[q]);
      } else if constexpr (HOUT) {
        dft_half_out<R, FWD>(v[q]);
      } else {
        dft<R, FWD>(v[q]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = t + q * T;
    if (PER * T == NB || b < NB) {
      const int j = (b / NS) * NS * R + (b % NS);
#pragma unroll
      for (int r = 0; r < ROUT; ++r) st(j + r * NS, v[q][r]);
    }
  }
  __syncthreads();
}

// Shared-memory view of one line: element p at base[p * STRIDE].
template <typename V, int STRIDE> struct SLine {
  V* base;
  __device__ __forceinline__ V get(int p) const { return base[p * STRIDE]; }
  __device__ __forceinline__ void put(int p, V v) const { base[p * STRIDE] = v; }
};

// Full transform of one line: stage 0 reads through `first`, the last stage
// writes through `last`, the stages in between go through the line view.
// HIN: the line's upper half (p >= M/2) is zero and `first` is only asked for
// p < M/2.  HOUT: only outputs p < M/2 are wanted; `last` sees only those
// (with an odd radix at that end the full stage runs instead).
template <class P, bool FWD, int T, typename V, bool HIN, bool HOUT, int S, class F, class L, class SL>
__device__ __forceinline__ void run_from(int t, const F& first, const L& last, const SL& sl) {
  auto sget = [&](int p) { return sl.get(p); };
  auto sput = [&](int p, V v) { sl.put(p, v); };
  if constexpr (S == 0 && P::NST == 1) {
    stage<P, 0, FWD, T, V, HIN, HOUT>(t, first, last);
  } else if constexpr (S == 0) {
    stage<P, 0, FWD, T, V, HIN, false>(t, first, sput);
    run_from<P, FWD, T, V, HIN, HOUT, 1>(t, first, last, sl);
  } else if constexpr (S == P::NST - 1) {
    stage<P, S, FWD, T, V, false, HOUT>(t, sget, last);
  } else {
    stage<P, S, FWD, T, V, false, false>(t, sget, sput);
    run_from<P, FWD, T, V, HIN, HOUT, S + 1>(t, first, last, sl);
  }
}

template <class P, bool FWD, int T, typename V, bool HIN = false, bool HOUT = false, class F, class L, class SL>
__device__ __forceinline__ void fft_line(int t, const F& first, const L& last, const SL& sl) {
  run_from<P, FWD, T, V, HIN, HOUT, 0>(t, first, last, sl);
}

}  // namespace fsa
