// Double-word (float-float) arithmetic for the FP64-accuracy tier.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, and the FP64 FFT
// passes are bound by that rate.  A double-word number hi + lo (two floats,
// |lo| <= ulp(hi)/2) carries 48 significand bits; its operations run on the
// FP32 pipes.  Building blocks (Joldes, Muller, Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", ACM TOMS
// 44(2), 2017):
//   TwoSum (Knuth), Fast2Sum (Dekker), 2Prod via FMA;
//   addition after "SloppyDWPlusDW" and multiplication after "DWTimesDW3"
//   (FMA based), each WITHOUT its closing Fast2Sum renormalisation.
// The result pair still represents hi + lo exactly; it is only not canonical
// (|lo| may exceed ulp(hi)/2).  After a cancellation most of a value can sit
// in lo, where later operations see it with float precision, but such a value
// is itself O(u |inputs|), so the absolute error stays O(u^2 |inputs|) -- the
// norm-wise bound an FFT's error analysis uses (u = 2^-24).  This saves 3 of
// 11 operations per addition and 3 of 9 per multiplication.
// Every float operation here goes through __fadd_rn / __fmul_rn / __fmaf_rn
// so the compiler can neither contract nor reorder it.
#pragma once
#include <cuda_runtime.h>

namespace fsa {

struct dw {
  float hi, lo;
  __host__ __device__ constexpr dw() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr dw(float h, float l) : hi(h), lo(l) {}
  // exact split of a double constant or value (rounded to 48 bits)
  __host__ __device__ constexpr dw(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr dw(int i) : hi((float)i), lo(0.f) {}
};

__device__ __forceinline__ dw dw_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dw(s, e);
}

__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return dw(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dw operator+(dw x, dw y) {
  const dw s = dw_two_sum(x.hi, y.hi);
  return dw(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dw operator-(dw x) { return dw(-x.hi, -x.lo); }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + dw(-y.hi, -y.lo); }

__device__ __forceinline__ dw operator*(dw x, dw y) {
  const float ch = __fmul_rn(x.hi, y.hi);
  const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
  const float tl0 = __fmul_rn(x.lo, y.lo);
  const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  return dw(ch, __fadd_rn(cl1, cl2));
}

// a * b + c * d: the two leading products exact (2Prod by FMA), summed by
// TwoSum, with the products' errors and the cross terms a.hi b.lo, a.lo b.hi,
// c.hi d.lo, c.lo d.hi folded in by FMA (a.lo b.lo and c.lo d.lo, of order
// u^2 |a b| and u^2 |c d|, are dropped).  16 operations against 20 for two
// multiplications and an addition; it carries the real and imaginary parts of
// a complex product.
__device__ __forceinline__ dw dw_dot2(dw a, dw b, dw c, dw d) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float pe = __fmaf_rn(a.hi, b.hi, -p);
  const float q = __fmul_rn(c.hi, d.hi);
  const float qe = __fmaf_rn(c.hi, d.hi, -q);
  const dw s = dw_two_sum(p, q);
  float t = __fadd_rn(pe, qe);
  t = __fmaf_rn(a.hi, b.lo, t);
  t = __fmaf_rn(a.lo, b.hi, t);
  t = __fmaf_rn(c.hi, d.lo, t);
  t = __fmaf_rn(c.lo, d.hi, t);
  return dw(s.hi, __fadd_rn(s.lo, t));
}

__device__ __forceinline__ dw dw_from_double(double d) {
  const float h = __double2float_rn(d);
  return dw(h, __double2float_rn(d - (double)h));
}
__device__ __forceinline__ double dw_to_double(dw x) { return (double)x.hi + (double)x.lo; }

// complex double-word: 16 bytes, like double2
struct __align__(16) cdw {
  dw x, y;
};

__device__ __forceinline__ cdw mk(dw x, dw y) {
  cdw r;
  r.x = x;
  r.y = y;
  return r;
}


}  // namespace fsa
