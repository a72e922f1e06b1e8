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

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// ---- paired form (sm_100 and later) -----------------------------------------
// A complex double-word value a = (a.x, a.y) as two register pairs: H = (a.x.hi,
// a.y.hi) and L = (a.x.lo, a.y.lo).  add/sub/mul/fma.rn.f32x2 apply one FP32
// operation to both halves of a pair, so each function below performs, for
// the real and the imaginary part at once, exactly the FP32 operations (same
// order, same rounding) of its scalar counterpart above.
typedef unsigned long long f2r;  // a register pair of two floats

__device__ __forceinline__ f2r p2(float a, float b) {
  f2r r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void u2(f2r r, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ f2r padd(f2r a, f2r b) {
  f2r r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2r psub(f2r a, f2r b) {
  f2r r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2r pmul(f2r a, f2r b) {
  f2r r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2r pfma(f2r a, f2r b, f2r c) {
  f2r r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ f2r hi2(cdw a) { return p2(a.x.hi, a.y.hi); }
__device__ __forceinline__ f2r lo2(cdw a) { return p2(a.x.lo, a.y.lo); }
__device__ __forceinline__ cdw from2(f2r h, f2r l) {
  cdw r;
  u2(h, r.x.hi, r.y.hi);
  u2(l, r.x.lo, r.y.lo);
  return r;
}

// TwoSum on pairs: s + e = a + b exactly, per half
__device__ __forceinline__ void pdw_two_sum(f2r a, f2r b, f2r& s, f2r& e) {
  s = padd(a, b);
  const f2r bb = psub(s, a);
  e = padd(psub(a, psub(s, bb)), psub(b, bb));
}

// a + b (operator+ on both parts)
__device__ __forceinline__ cdw dwp_add(cdw a, cdw b) {
  f2r s, e;
  pdw_two_sum(hi2(a), hi2(b), s, e);
  return from2(s, padd(e, padd(lo2(a), lo2(b))));
}
// a - b = a + (-b) (operator- on both parts).  TwoSum(a, -b) written with
// subtractions: s = a - b, bb = s - a, e = (a - (s - bb)) - (b + bb); each
// step is the negation-free twin of TwoSum's, rounded identically.
__device__ __forceinline__ cdw dwp_sub(cdw a, cdw b) {
  const f2r ah = hi2(a), bh = hi2(b);
  const f2r s = psub(ah, bh);
  const f2r bb = psub(s, ah);
  const f2r e = psub(psub(ah, psub(s, bb)), padd(bh, bb));
  return from2(s, padd(e, psub(lo2(a), lo2(b))));
}
// a * s for a real double-word s (operator* on both parts).  The product's
// error cl1 = fma(a.hi, s.hi, -ch) is formed negated, fma(a.hi, -s.hi, ch),
// and subtracted at the end: the same roundings, no negation instruction.
__device__ __forceinline__ cdw dwp_scale(cdw a, dw s) {
  const f2r sh = p2(s.hi, s.hi), nsh = p2(-s.hi, -s.hi), sl = p2(s.lo, s.lo), ah = hi2(a), al = lo2(a);
  const f2r ch = pmul(ah, sh);
  const f2r ncl1 = pfma(ah, nsh, ch);
  const f2r tl0 = pmul(al, sl);
  const f2r tl1 = pfma(ah, sl, tl0);
  const f2r cl2 = pfma(al, sh, tl1);
  return from2(ch, psub(cl2, ncl1));
}
// a * b (CONJ: a * conj(b)) with both parts as dw_dot2: the real part
// a.x b.x - a.y b.y and the imaginary part a.x b.y + a.y b.x (conjugate:
// a.x b.x + a.y b.y and a.y b.x - a.x b.y) share their operand pattern
// c1 * d1 + c2 * d2 with c = broadcast parts of a and d = parts of b.
template <bool CONJ> __device__ __forceinline__ cdw dwp_cmul(cdw a, cdw b) {
  // dot2 operands per half (real, imaginary):
  //   plain: (a.x, a.x) * (b.x, b.y) + (a.y, a.y) * (-b.y, b.x)
  //   conj:  (a.x, a.y) * (b.x, b.x) + (a.y, a.x) * (b.y, -b.y)
  f2r c1h, c1l, d1h, d1l, c2h, c2l, d2h, d2l;
  if (CONJ) {
    c1h = p2(a.x.hi, a.y.hi); c1l = p2(a.x.lo, a.y.lo);
    d1h = p2(b.x.hi, b.x.hi); d1l = p2(b.x.lo, b.x.lo);
    c2h = p2(a.y.hi, a.x.hi); c2l = p2(a.y.lo, a.x.lo);
    d2h = p2(b.y.hi, -b.y.hi); d2l = p2(b.y.lo, -b.y.lo);
  } else {
    c1h = p2(a.x.hi, a.x.hi); c1l = p2(a.x.lo, a.x.lo);
    d1h = p2(b.x.hi, b.y.hi); d1l = p2(b.x.lo, b.y.lo);
    c2h = p2(a.y.hi, a.y.hi); c2l = p2(a.y.lo, a.y.lo);
    d2h = p2(-b.y.hi, b.x.hi); d2l = p2(-b.y.lo, b.x.lo);
  }
  const f2r m1 = p2(-1.f, -1.f);
  const f2r p = pmul(c1h, d1h);
  const f2r pe = pfma(c1h, d1h, pmul(p, m1));
  const f2r q = pmul(c2h, d2h);
  const f2r qe = pfma(c2h, d2h, pmul(q, m1));
  f2r s, e;
  pdw_two_sum(p, q, s, e);
  f2r t = padd(pe, qe);
  t = pfma(c1h, d1l, t);
  t = pfma(c1l, d1h, t);
  t = pfma(c2h, d2l, t);
  t = pfma(c2l, d2h, t);
  return from2(s, padd(e, t));
}
// canonical form: one TwoSum per part
__device__ __forceinline__ cdw dwp_canon(cdw v) {
  f2r s, e;
  pdw_two_sum(hi2(v), lo2(v), s, e);
  return from2(s, e);
}
#endif

}  // namespace fsa
