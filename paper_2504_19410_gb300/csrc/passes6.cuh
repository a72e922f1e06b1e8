// Sixth-generation FP32 middle pass: the axis-1 forward transform, the
// multiply by the real, even spectrum and the inverse transform of the
// second generation (passes2.cuh: M = R1 x R2 in two register-resident steps,
// the multiply between forward and inverse step B), with half the values per
// thread, so that twice as many warps fit on an SM.
//
// The second generation's step A holds one whole length-R1 sub-transform per
// thread (R1 complex values).  Its input is half zero (the padding) and, in
// the inverse, half of its output is discarded (the crop), so it splits into
// two independent halves of length R1/2:
//   forward (half-zero input x_r, r < R1/2):
//     A[2j]     = DFT_{R1/2}(x_r)[j]            (half h = 0)
//     A[2j + 1] = DFT_{R1/2}(x_r w_R1^r)[j]     (half h = 1)
//   inverse (outputs r < R1/2 kept):
//     x[r] = IDFT_{R1/2}(A[2j])[r] + w_R1^-r IDFT_{R1/2}(A[2j + 1])[r]
// Here each half is a task of its own thread: R1/2 values.  Forward, the two
// halves go to different exchange slots and need nothing from each other.
// Inverse, the two partial sums of x[r] meet through a small shared-memory
// buffer: the task of half h keeps the outputs r in [h R1/4, (h+1) R1/4) and
// hands the other quarter of its partial sums to its partner.  With
// R1 = 2 R2 every thread has one step-A task and one step-B sub-transform of
// R2 values (512 = 32 x 16: 16 values, against 32 in the second generation).
//
// Lanes: l = column (threadIdx % 16); the thread's group g = threadIdx / 16
// gives its step-A tasks (a = g + R1 i: t = a mod R2, h = a / R2, so h is the
// same across a warp and the half's branch never diverges) and, through
// mid_u, its step-B sub-transform q (the threads holding k1 and M - k1 share a
// warp: one spectrum load per pair and a shuffle, as in passes2.cuh).  The
// launch bounds ask for 24 to 32 resident warps per SM (Plan6::MINB).
// Three barriers per tile: after step A, after step B, after the partial
// sums are handed over.  The inputs are loaded straight from HBM: the
// resident warps hide the latency.
#pragma once
#include "passes2.cuh"

namespace fsa {

template <int M_, int R1_, int R2_> struct Plan6 {
  static constexpr int M = M_, R1 = R1_, R2 = R2_, T = R1_;
  static constexpr int H = R1 / 2;               // values of a step-A half task
  static constexpr int Q = R1 / 4;               // outputs a half task keeps
  static constexpr int TASKS = 2 * R2;           // step-A half tasks per line
  static constexpr int PA = (TASKS + R1 - 1) / R1;
  static constexpr int W = 16;                   // columns per CTA
  static constexpr int NT = W * R1;
  static constexpr int EX = M * W;               // exchange tile (complex values)
  static constexpr int CB = TASKS * Q * W;       // hand-over buffer (complex values)
  static constexpr int SMEM = (EX + CB) * 8;
  // resident CTAs asked of the compiler: 32 warps per SM (64 registers) for
  // 512-thread CTAs; 3 CTAs (85 registers) for 256-thread CTAs, whose
  // length-8 and length-12/16 transforms spill at 64
  static constexpr int MINB = NT >= 512 ? 2 : 3;
  static_assert(R1 * R2 == M && R1 % 4 == 0 && R2 % 2 == 0, "plan factors");
  // the warp-uniform half index needs the two groups of a warp in one half
  static_assert(R2 % 2 == 0 && (PA == 1 || R1 % R2 == 0 || R2 % 2 == 0), "half index per warp");
};

template <int M> struct Plan6For;
template <> struct Plan6For<128> { using type = Plan6<128, 16, 8>; };
template <> struct Plan6For<192> { using type = Plan6<192, 16, 12>; };
template <> struct Plan6For<256> { using type = Plan6<256, 16, 16>; };
template <> struct Plan6For<384> { using type = Plan6<384, 16, 24>; };
template <> struct Plan6For<512> { using type = Plan6<512, 32, 16>; };

template <class P>
__global__ void __launch_bounds__(P::NT, P::MINB) k6_col_mid(const Jobs jobs, int M2, int planes) {
  using V = float2;
  constexpr int M = P::M, n = M / 2, W = P::W, R1 = P::R1, R2 = P::R2, H = P::H, Q = P::Q, PA = P::PA;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* ex = reinterpret_cast<V*>(smraw);  // [q][t][l], q < R1, t < R2
  V* cb = ex + P::EX;                   // [t][h][i][l], i < Q: sums handed to task (t, h)
  const int l = threadIdx.x % W, g = threadIdx.x / W;
  const int u = mid_u<P>(threadIdx.x);  // step-B sub-transform of this thread
  const int tiles_per_plane = (M2 + W - 1) / W;
  const long long tpj = (long long)tiles_per_plane * planes;
  const int n2 = M2 / 2;
  for (long long tile = blockIdx.x; tile < tpj * jobs.count; tile += gridDim.x) {
    const Job& jb = jobs.j[tile / tpj];
    const int lt = (int)(tile % tpj);
    const int k0 = lt / tiles_per_plane;
    const int k2 = (lt % tiles_per_plane) * W + l;
    const bool ok = k2 < M2;
    V* __restrict__ col = static_cast<V*>(jb.out) + (long long)k0 * n * M2 + (ok ? k2 : 0);
    const float* __restrict__ srow =
        static_cast<const float*>(jb.S) + (long long)k0 * (n + 1) * (n2 + 1) + (ok ? min(k2, M2 - k2) : 0);
    // step A, forward: task (t, h) -> A[2j + h] w_M^{t (2j + h)} at slot (2j + h, t)
#pragma unroll
    for (int i = 0; i < PA; ++i) {
      const int a = g + R1 * i;
      if (P::TASKS % R1 == 0 || a < P::TASKS) {
        const int t = a % R2, h = a / R2;
        V x[H];
#pragma unroll
        for (int r = 0; r < H; ++r) x[r] = ok ? col[(long long)(t + R2 * r) * M2] : czero<V>();
        if (h) {
          sfor<1, H>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            x[r] = twc<R1, r, true>(x[r]);
          });
        }
        rfft<H, true>(x);
#pragma unroll
        for (int j = 0; j < H; ++j) {
          const int q = 2 * j + h;
          ex[(q * R2 + t) * W + l] = cmul(x[j], twiddle<V, M>(t * q));
        }
      }
    }
    __syncthreads();
    // step B: forward length-R2 transform, spectrum, inverse, twiddles back
    MidSpec<P> sp;
    mid_load<P>(sp, srow, u, ok, n2 + 1);
    V b[R2];
#pragma unroll
    for (int t = 0; t < R2; ++t) b[t] = ex[(u * R2 + t) * W + l];
    rfft<R2, true>(b);
    mid_apply<P>(b, sp, u);
    // the slots this thread read are the ones it writes: no barrier needed
    stepB_inv<P, V>(u, b, [&](int q, int t, V v) { ex[(q * R2 + t) * W + l] = v; });
    __syncthreads();
    // step A, inverse: task (t, h) forms IDFT(A[2j + h]) (times w_R1^-r for
    // h = 1), keeps r in [h Q, h Q + Q) and hands the other quarter over
    V z[PA][H];
#pragma unroll
    for (int i = 0; i < PA; ++i) {
      const int a = g + R1 * i;
      if (P::TASKS % R1 == 0 || a < P::TASKS) {
        const int t = a % R2, h = a / R2;
#pragma unroll
        for (int j = 0; j < H; ++j) z[i][j] = ex[((2 * j + h) * R2 + t) * W + l];
        rfft<H, false>(z[i]);
        if (h) {
          sfor<1, H>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            z[i][r] = twc<R1, r, false>(z[i][r]);
          });
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) cb[((t * 2 + (1 - h)) * Q + k) * W + l] = h ? z[i][k] : z[i][Q + k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PA; ++i) {
      const int a = g + R1 * i;
      if (P::TASKS % R1 == 0 || a < P::TASKS) {
        const int t = a % R2, h = a / R2;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
          const V own = h ? z[i][Q + k] : z[i][k];
          const V v = cadd(own, cb[((t * 2 + h) * Q + k) * W + l]);
          if (ok) col[(long long)(t + R2 * (h * Q + k)) * M2] = v;
        }
      }
    }
    // the next tile's step A writes only ex, which every thread has finished
    // reading (before the last barrier); cb is next written after two more
  }
}

}  // namespace fsa
