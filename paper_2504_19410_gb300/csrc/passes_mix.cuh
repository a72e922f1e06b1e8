// Mixed-length FP32 apply passes: one persistent launch per pass over the
// concatenated tile lists of many solves whose grids differ.
//
// A batch of solves of uneven n (Sec. 2.3's five passes per solve) would need
// one launch per pass and transform length.  Here each pass is ONE launch:
// the host lists every solve's tiles back to back (MixJobs.begin holds the
// prefix sums), a CTA walks tiles grid-stride, finds the tile's solve and
// runs the tile body compiled for that solve's transform length (a switch
// over the lengths the kernel carries).  Every length uses the same thread
// geometry, M = 16 x (M / 16) (R1 = 16 threads per line, W = 16 lines or
// columns per CTA, 256 threads), so one block shape and one shared-memory
// size serve all of them.  The tile bodies are the second-generation
// register transforms (passes2.cuh) with the same loads, exchanges and
// stores; every body ends with a barrier, so consecutive tiles of different
// lengths can reuse the shared memory.
#pragma once
#include "passes2.cuh"

namespace fsa {

// One solve of a mixed launch: in / out / spectrum of the pass, and its grid.
struct MixJob {
  const void* in;
  void* out;
  const void* S;
  int n0, n1, n2;
};
struct MixJobs {
  MixJob j[kMaxJobs];
  long long begin[kMaxJobs + 1];  // first tile of solve k; begin[count] = all tiles
  int count;
};

enum MixPass { kMixR2C = 0, kMixRowF = 1, kMixCol = 2, kMixRowI = 3, kMixC2R = 4 };

template <int M> using MixPlan = Plan2<M, 16, M / 16>;
constexpr int kMixW = 16, kMixNT = 256;
// shared memory of the largest length a mixed launch carries
__host__ __device__ constexpr int mix_smem(int M) {
  return (M * kMixW > kMixW * 16 * (M / 16 + 1) ? M * kMixW : kMixW * 16 * (M / 16 + 1)) * 8;
}

// Tiles of one solve for a pass (host and device agree on these).
__host__ __device__ inline long long mix_tiles(int pass, int n0, int n1, int n2) {
  const long long C = (long long)n1 * n2, rows = (long long)(n0 + 1) * n1;
  switch (pass) {
    case kMixR2C:
    case kMixC2R: return (C + 2 * kMixW - 1) / (2 * kMixW);
    case kMixRowF:
    case kMixRowI: return (rows + kMixW - 1) / kMixW;
    default: return (long long)((2 * n2 + kMixW - 1) / kMixW) * (n0 + 1);
  }
}

template <class P> __device__ __forceinline__ void mix_r2c(const MixJob& jb, long long lt, float2* sm) {
  using V = float2;
  constexpr int M = P::M, n = M / 2, K = M / 2 + 1, W = kMixW, R1 = P::R1, R2 = P::R2;
  const int l = threadIdx.x % W, u = threadIdx.x / W;
  const long long C = (long long)jb.n1 * jb.n2;
  const float* __restrict__ rho = static_cast<const float*>(jb.in);
  V* __restrict__ X = static_cast<V*>(jb.out);
  const long long c = lt * (2 * W) + 2 * l;
  const bool ok = c < C;
  stepA_fwd<P, V, true>(
      u,
      [&](int t, int r) {
        const int p = t + R2 * r;
        return (p < n && ok) ? *reinterpret_cast<const V*>(rho + (long long)p * C + c) : czero<V>();
      },
      [&](int q, int t, V v) { sm[(q * R2 + t) * W + l] = v; });
  __syncthreads();
  V b[R2];
#pragma unroll
  for (int t = 0; t < R2; ++t) b[t] = sm[(u * R2 + t) * W + l];
  rfft<R2, true>(b);
  __syncthreads();
#pragma unroll
  for (int s = 0; s < R2; ++s) sm[(u + R1 * s) * W + l] = b[s];
  __syncthreads();
  // two real columns as one complex line: A[k] = (Z[k] + conj Z[M-k]) / 2,
  // B[k] = (Z[k] - conj Z[M-k]) / 2i
  for (int k = u; k < K; k += P::T) {
    const V zk = sm[k * W + l];
    const V zm = sm[((M - k) % M) * W + l];
    if (ok)
      *reinterpret_cast<float4*>(X + (long long)k * C + c) =
          make_float4(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y), 0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
  }
  __syncthreads();
}

template <class P> __device__ __forceinline__ void mix_row_fwd(const MixJob& jb, long long lt, float2* sm) {
  using V = float2;
  constexpr int M = P::M, n = M / 2, W = kMixW, R1 = P::R1, R2 = P::R2, PITCH = P::R1 * (P::R2 + 1);
  const int u = threadIdx.x % P::T, l = threadIdx.x / P::T;
  V* line = sm + l * PITCH;
  const long long rows = (long long)(jb.n0 + 1) * jb.n1;
  const long long row = lt * W + l;
  const bool ok = row < rows;
  const V* __restrict__ x = static_cast<const V*>(jb.in) + (ok ? row * n : 0);
  V* __restrict__ y = static_cast<V*>(jb.out) + (ok ? row * M : 0);
  stepA_fwd<P, V, true>(
      u,
      [&](int t, int r) {
        const int p = t + R2 * r;
        return (p < n && ok) ? x[p] : czero<V>();
      },
      [&](int q, int t, V v) { line[q * (R2 + 1) + t] = v; });
  __syncthreads();
  V b[R2];
#pragma unroll
  for (int t = 0; t < R2; ++t) b[t] = line[u * (R2 + 1) + t];
  rfft<R2, true>(b);
  if (ok) {
#pragma unroll
    for (int s = 0; s < R2; ++s) y[u + R1 * s] = b[s];
  }
  __syncthreads();
}

template <class P> __device__ __forceinline__ void mix_col(const MixJob& jb, long long lt, float2* sm) {
  using V = float2;
  constexpr int M = P::M, n = M / 2, W = kMixW, R1 = P::R1, R2 = P::R2;
  const int l = threadIdx.x % W, u = mid_u<P>(threadIdx.x);
  const int M2 = 2 * jb.n2, n2 = jb.n2;
  const int tiles_per_plane = (M2 + W - 1) / W;
  const int k0 = (int)(lt / tiles_per_plane);
  const int k2 = (int)(lt % tiles_per_plane) * W + l;
  const bool ok = k2 < M2;
  V* __restrict__ col = static_cast<V*>(jb.out) + (long long)k0 * n * M2 + (ok ? k2 : 0);
  const float* __restrict__ srow =
      static_cast<const float*>(jb.S) + (long long)k0 * (n + 1) * (n2 + 1) + (ok ? min(k2, M2 - k2) : 0);
  stepA_fwd<P, V, true>(
      u,
      [&](int t, int r) {
        const int p = t + R2 * r;
        return (p < n && ok) ? col[(long long)p * M2] : czero<V>();
      },
      [&](int q, int t, V v) { sm[(q * R2 + t) * W + l] = v; });
  __syncthreads();
  MidSpec<P> sp;
  mid_load<P>(sp, srow, u, ok, n2 + 1);
  V b[R2];
#pragma unroll
  for (int t = 0; t < R2; ++t) b[t] = sm[(u * R2 + t) * W + l];
  rfft<R2, true>(b);
  mid_apply<P>(b, sp, u);
  stepB_inv<P, V>(u, b, [&](int q, int t, V v) { sm[(q * R2 + t) * W + l] = v; });
  __syncthreads();
  stepA_inv<P, V, true>(
      u, [&](int q, int t) { return sm[(q * R2 + t) * W + l]; },
      [&](int t, int r, V v) {
        const int p = t + R2 * r;
        if (p < n && ok) col[(long long)p * M2] = v;
      });
  __syncthreads();
}

template <class P> __device__ __forceinline__ void mix_row_inv(const MixJob& jb, long long lt, float2* sm) {
  using V = float2;
  constexpr int M = P::M, n = M / 2, W = kMixW, R1 = P::R1, R2 = P::R2, PITCH = P::R1 * (P::R2 + 1);
  const int u = threadIdx.x % P::T, l = threadIdx.x / P::T;
  V* line = sm + l * PITCH;
  const long long rows = (long long)(jb.n0 + 1) * jb.n1;
  const long long row = lt * W + l;
  const bool ok = row < rows;
  const V* __restrict__ y = static_cast<const V*>(jb.in) + (ok ? row * M : 0);
  V* __restrict__ x = static_cast<V*>(jb.out) + (ok ? row * n : 0);
  V b[R2];
#pragma unroll
  for (int s = 0; s < R2; ++s) b[s] = ok ? y[u + R1 * s] : czero<V>();
  stepB_inv<P, V>(u, b, [&](int q, int t, V v) { line[q * (R2 + 1) + t] = v; });
  __syncthreads();
  stepA_inv<P, V, true>(
      u, [&](int q, int t) { return line[q * (R2 + 1) + t]; },
      [&](int t, int r, V v) {
        const int p = t + R2 * r;
        if (p < n && ok) x[p] = v;
      });
  __syncthreads();
}

template <class P> __device__ __forceinline__ void mix_c2r(const MixJob& jb, long long lt, float2* sm) {
  using V = float2;
  constexpr int M = P::M, n = M / 2, W = kMixW, R1 = P::R1, R2 = P::R2;
  const int l = threadIdx.x % W, u = threadIdx.x / W;
  const long long C = (long long)jb.n1 * jb.n2;
  const V* __restrict__ X = static_cast<const V*>(jb.in);
  float* __restrict__ phi = static_cast<float*>(jb.out);
  const long long c = lt * (2 * W) + 2 * l;
  const bool ok = c < C;
  // Z[k] = A[k] + i B[k] with A, B Hermitian: rebuild k > n from M - k
  V b[R2];
#pragma unroll
  for (int s = 0; s < R2; ++s) {
    const int k = u + R1 * s;
    V z = czero<V>();
    if (ok) {
      const bool lo = k <= n;
      const long long kk = lo ? k : M - k;
      const float4 ab = *reinterpret_cast<const float4*>(X + kk * C + c);
      z = lo ? mk(ab.x - ab.w, ab.y + ab.z) : mk(ab.x + ab.w, ab.z - ab.y);
    }
    b[s] = z;
  }
  stepB_inv<P, V>(u, b, [&](int q, int t, V v) { sm[(q * R2 + t) * W + l] = v; });
  __syncthreads();
  stepA_inv<P, V, true>(
      u, [&](int q, int t) { return sm[(q * R2 + t) * W + l]; },
      [&](int t, int r, V v) {
        const int p = t + R2 * r;
        if (p < n && ok) *reinterpret_cast<V*>(phi + (long long)p * C + c) = v;
      });
  __syncthreads();
}

template <int PASS, int M> __device__ __forceinline__ void mix_tile(const MixJob& jb, long long lt, float2* sm) {
  using P = MixPlan<M>;
  if constexpr (PASS == kMixR2C) mix_r2c<P>(jb, lt, sm);
  else if constexpr (PASS == kMixRowF) mix_row_fwd<P>(jb, lt, sm);
  else if constexpr (PASS == kMixCol) mix_col<P>(jb, lt, sm);
  else if constexpr (PASS == kMixRowI) mix_row_inv<P>(jb, lt, sm);
  else mix_c2r<P>(jb, lt, sm);
}

// Transform length of a solve's pass: axis 0 for the R2C / C2R passes, axis 2
// for the row passes, axis 1 for the middle pass.
__host__ __device__ inline int mix_length(int pass, int n0, int n1, int n2) {
  return 2 * (pass == kMixR2C || pass == kMixC2R ? n0 : (pass == kMixCol ? n1 : n2));
}

// The lengths a mixed launch carries: the cubic grids 64^3 ... 256^3 of the
// batched workload (M = 2n = 128, 192, 256, 384, 512).
__host__ __device__ constexpr bool mix_supported(int M) {
  return M == 128 || M == 192 || M == 256 || M == 384 || M == 512;
}

template <int PASS> __device__ __forceinline__ void mix_dispatch(const MixJob& jb, long long lt, float2* sm) {
  switch (mix_length(PASS, jb.n0, jb.n1, jb.n2)) {
    case 128: mix_tile<PASS, 128>(jb, lt, sm); break;
    case 192: mix_tile<PASS, 192>(jb, lt, sm); break;
    case 256: mix_tile<PASS, 256>(jb, lt, sm); break;
    case 384: mix_tile<PASS, 384>(jb, lt, sm); break;
    default: mix_tile<PASS, 512>(jb, lt, sm); break;
  }
}

// Two passes of two halves of a batch in one launch (software pipelining:
// half A's pass PA beside half B's pass PB, whose inputs are ready): the two
// tile lists are interleaved tile by tile, so the CTAs on an SM run tiles of
// both passes at once -- the middle pass, bound by its arithmetic, beside a
// row pass, bound by HBM.
template <int PA, int PB>
__global__ void __launch_bounds__(kMixNT, 2) k_mix2(const MixJobs a, const MixJobs b) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const long long ta = a.begin[a.count], tb = b.begin[b.count], both = ta < tb ? ta : tb;
  const long long total = ta + tb;
  int ka = 0, kb = 0;
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
    // tile -> (list, index): alternate while both lists last, then the longer one
    bool in_a;
    long long i;
    if (tile < 2 * both) {
      in_a = (tile & 1) == 0;
      i = tile >> 1;
    } else {
      in_a = ta > tb;
      i = tile - both;
    }
    if (in_a) {
      while (i >= a.begin[ka + 1]) ++ka;
      mix_dispatch<PA>(a.j[ka], i - a.begin[ka], sm);
    } else {
      while (i >= b.begin[kb + 1]) ++kb;
      mix_dispatch<PB>(b.j[kb], i - b.begin[kb], sm);
    }
  }
}

template <int PASS>
__global__ void __launch_bounds__(kMixNT, 2) k_mix(const MixJobs js) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const long long total = js.begin[js.count];
  int k = 0;
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
    while (tile >= js.begin[k + 1]) ++k;  // tiles only increase: the solve index only grows
    const MixJob& jb = js.j[k];
    const long long lt = tile - js.begin[k];
    switch (mix_length(PASS, jb.n0, jb.n1, jb.n2)) {
      case 128: mix_tile<PASS, 128>(jb, lt, sm); break;
      case 192: mix_tile<PASS, 192>(jb, lt, sm); break;
      case 256: mix_tile<PASS, 256>(jb, lt, sm); break;
      case 384: mix_tile<PASS, 384>(jb, lt, sm); break;
      default: mix_tile<PASS, 512>(jb, lt, sm); break;
    }
  }
}

}  // namespace fsa
