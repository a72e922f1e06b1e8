// Second-generation apply passes: the same five passes and data flow as
// passes.cuh (pad + R2C axis 0 -> axis-2 FFT -> axis-1 FFT x spectrum x
// inverse -> axis-2 inverse -> C2R axis 0 + crop), with every line transformed
// as M = R1 x R2 in two register-resident steps (fft_reg.cuh).  Shared-memory
// exchanges per line: R2C 2, row forward 1, middle 2, row inverse 1, C2R 1
// (the first generation needed 3-5 per pass).
//
// Strided passes (axes 0, 1): W lines per CTA, lanes on lines, so each warp
// access to HBM covers W consecutive elements of the contiguous axis; the
// shared tile is sm[p * W + l].  Row passes (axis 2): lanes on the R1 threads
// of a line, so step A's loads x[t + R2 r] and step B's stores X[q + R1 s]
// are contiguous per half-warp; the shared tile is sm[l * R1 (R2+1) + q (R2+1) + t]
// (padded rows: conflict-free for both steps).
#pragma once
#include "ddi.cuh"
#include "fft_reg.cuh"

namespace fsa {

template <class P> struct Geo2 {
  static constexpr int W = 16;
  static constexpr int NT = W * P::T;
  // the middle pass asks for two resident CTAs (<= 128 registers) when a CTA
  // has at most 256 threads
  static constexpr int MINB_MID = NT <= 256 ? 2 : 1;
  // the R2C pass holds fewer live values: three resident CTAs when small
  // (measured faster; the row passes and C2R measured slower so capped)
  static constexpr int MINB = NT <= 256 ? 3 : 1;
  static constexpr int SM_STRIDED = P::M * W * 8;
  static constexpr int PITCH = P::R1 * (P::R2 + 1);
  static constexpr int SM_ROWS = W * PITCH * 8;
};

// ---------------------------------------------------------------- pass 1 --
// PAD = false: the unpadded transform over all M inputs (the DDI grid
// reading), same K = M/2 + 1 outputs.
template <class P, bool PAD = true>
__global__ void __launch_bounds__(Geo2<P>::NT, Geo2<P>::MINB) k2_r2c_ax0(const Jobs jobs, long long C) {
  using V = float2;
  constexpr int M = P::M, n = PAD ? M / 2 : M, K = M / 2 + 1, W = Geo2<P>::W, R1 = P::R1, R2 = P::R2;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int l = threadIdx.x % W, u = threadIdx.x / W;
  const long long tpj = (C + 2 * W - 1) / (2 * W);
  for (long long tile = blockIdx.x; tile < tpj * jobs.count; tile += gridDim.x) {
    const Job& jb = jobs.j[tile / tpj];
    const float* __restrict__ rho = static_cast<const float*>(jb.in);
    V* __restrict__ X = static_cast<V*>(jb.out);
    const long long c = (tile % tpj) * (2 * W) + 2 * l;
    const bool ok = c < C;
    stepA_fwd<P, V, PAD>(
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
    // Z = DFT(a + i b): A[k] = (Z[k] + conj Z[M-k]) / 2, B[k] = (Z[k] - conj Z[M-k]) / 2i
    for (int k = u; k < K; k += P::T) {
      const V zk = sm[k * W + l];
      const V zm = sm[((M - k) % M) * W + l];
      if (ok) {
        // columns c and c + 1 are adjacent (c even, C even): one 16-byte store
        *reinterpret_cast<float4*>(X + (long long)k * C + c) =
            make_float4(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y), 0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- pass 2 --
template <class P>
__global__ void __launch_bounds__(Geo2<P>::NT) k2_row_fwd(const Jobs jobs, long long rows) {
  using V = float2;
  constexpr int M = P::M, n = M / 2, W = Geo2<P>::W, R1 = P::R1, R2 = P::R2, PITCH = Geo2<P>::PITCH;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int u = threadIdx.x % P::T, l = threadIdx.x / P::T;
  V* line = sm + l * PITCH;
  const long long tpj = (rows + W - 1) / W;
  for (long long tile = blockIdx.x; tile < tpj * jobs.count; tile += gridDim.x) {
    const Job& jb = jobs.j[tile / tpj];
    const long long row = (tile % tpj) * W + l;
    const bool ok = row < rows;
    const V* __restrict__ x = static_cast<const V*>(jb.in) + row * n;
    V* __restrict__ y = static_cast<V*>(jb.out) + row * M;
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
}

// ---------------------------------------------------------------- pass 3 --
// Lanes of the middle pass: l = column (threadIdx % W), u = sub-transform
// index.  With R1 even, the two half-warps of warp w hold u = w and its
// mirror R1 - w (warp 0: u = 0 and R1/2, each its own mirror), so that the
// spectrum values of k1 and M - k1 -- equal, the spectrum is even -- take one
// load and a shuffle (mid_scale).
template <class P> __device__ __forceinline__ int mid_u(int tid) {
  constexpr int R1 = P::R1;
  if constexpr (R1 % 2 == 0 && P::R2 % 2 == 0 && Geo2<P>::W == 16) {
    const int w = tid >> 5, h = (tid >> 4) & 1;
    return h == 0 ? w : (w == 0 ? R1 / 2 : R1 - w);
  } else {
    return tid / Geo2<P>::W;
  }
}

// The spectrum values S(k1) of one thread, k1 = u + R1 s (s < R2), with
// S(k1) = srow[min(k1, M - k1) st].  mid_load issues the loads (so their
// latency can pass under the forward transform), mid_apply multiplies.
template <class P> struct MidSpec {
  static constexpr bool PAIRED = P::R1 % 2 == 0 && P::R2 % 2 == 0 && Geo2<P>::W == 16;
  static constexpr int NV = PAIRED ? P::R2 / 2 + 1 : P::R2;  // paired: s < R2/2, then the Nyquist value
  float v[NV];
};

template <class P>
__device__ __forceinline__ void mid_load(MidSpec<P>& sp, const float* __restrict__ srow, int u, bool ok, int st) {
  constexpr int M = P::M, R1 = P::R1, R2 = P::R2, H = R2 / 2;
  const float* lo = srow + u * st;
  if constexpr (MidSpec<P>::PAIRED) {
    // k1 < M/2 for s < R2/2: this thread's own loads; v[H] = S(M/2) for u = 0
#pragma unroll
    for (int s = 0; s < H; ++s) sp.v[s] = ok ? __ldg(lo + (R1 * s) * st) : 0.f;
    sp.v[H] = (ok && (threadIdx.x >> 5) == 0) ? __ldg(srow + (M / 2) * st) : 0.f;
  } else {
    // the even spectrum's index min(k1, M - k1) is k1 for s < R2/2 and M - k1
    // from s = R2/2 on (u < R1), decided at compile time
    const float* hi = srow + (M - u) * st;
#pragma unroll
    for (int s = 0; s < R2; ++s) sp.v[s] = !ok ? 0.f : (2 * s < R2 ? __ldg(lo + (R1 * s) * st) : __ldg(hi - (R1 * s) * st));
  }
}

// f(s, S) turns the spectrum value of element s (k1 = u + R1 s) into the
// value that multiplies it (the identity for the plain spectrum multiply).
struct SpecOnly {
  __device__ __forceinline__ float operator()(int, float v) const { return v; }
};

template <class P, class F = SpecOnly>
__device__ __forceinline__ void mid_apply(float2* b, const MidSpec<P>& sp, int u, F f = F()) {
  constexpr int R1 = P::R1, R2 = P::R2, H = R2 / 2;
  if constexpr (MidSpec<P>::PAIRED) {
#pragma unroll
    for (int s = 0; s < H; ++s) b[s] = cscale(b[s], f(s, sp.v[s]));
    // s >= R2/2: S(M - k1) with M - k1 = (R1 - u) + R1 (R2 - 1 - s) for u > 0
    if ((threadIdx.x >> 5) == 0) {  // u = 0 (M - k1 = R1 (R2 - s); Nyquist at s = R2/2) or u = R1/2
      sfor<H, R2>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        const float a = sp.v[s == H ? H : R2 - s];
        b[s] = cscale(b[s], f(s, u == 0 ? a : sp.v[R2 - 1 - s]));
      });
    } else {  // the mirror u' = R1 - u is the other half of this warp
#pragma unroll
      for (int s = H; s < R2; ++s) b[s] = cscale(b[s], f(s, __shfl_xor_sync(0xffffffffu, sp.v[R2 - 1 - s], 16)));
    }
  } else {
#pragma unroll
    for (int s = 0; s < R2; ++s) b[s] = cscale(b[s], f(s, sp.v[s]));
  }
}

// The middle pass's multiply: the spectrum alone, or (kMulDdiKernel) the 3-D
// DDI kernel reading's cmul * S * D + cadd at k1 = u + R1 s.
template <class P, int MODE>
__device__ __forceinline__ void mid_multiply(float2* b, const MidSpec<P>& sp, int u, const Job& jb, int k0, int k2,
                                             int M2, bool ok) {
  if constexpr (MODE == kMulSpectrum) {
    mid_apply<P>(b, sp, u);
  } else if constexpr (MODE == kMulDdiKernel) {
    DdiLine<float2> ddi;
    ddi.init(jb.par, k0, ok ? k2 : 0, M2);
    mid_apply<P>(b, sp, u, [&](int s, float v) { return ddi.template value<MODE>(v, u + P::R1 * s, P::M); });
  } else {  // kMulDdiGrid: no spectrum
    DdiLine<float2> ddi;
    ddi.init(jb.par, k0, ok ? k2 : 0, M2);
#pragma unroll
    for (int s = 0; s < P::R2; ++s) b[s] = cscale(b[s], ddi.template value<MODE>(0.f, u + P::R1 * s, P::M));
  }
}

template <class P, int MODE = kMulSpectrum>
__global__ void __launch_bounds__(Geo2<P>::NT, Geo2<P>::MINB_MID) k2_col_mid(const Jobs jobs, int M2, int planes) {
  using V = float2;
  constexpr bool PAD = MODE != kMulDdiGrid;
  constexpr int M = P::M, n = PAD ? M / 2 : M, W = Geo2<P>::W, R1 = P::R1, R2 = P::R2;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int l = threadIdx.x % W, u = mid_u<P>(threadIdx.x);
  const int tiles_per_plane = (M2 + W - 1) / W;
  const long long tpj = (long long)tiles_per_plane * planes;
  const int n2 = M2 / 2;
  const long long total = tpj * jobs.count;
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const long long tile = kMidReverse ? total - 1 - it : it;
    const Job& jb = jobs.j[tile / tpj];
    const int lt = (int)(tile % tpj);
    const int k0 = lt / tiles_per_plane;
    const int k2 = (lt % tiles_per_plane) * W + l;
    const bool ok = k2 < M2;
    V* __restrict__ col = static_cast<V*>(jb.out) + (long long)k0 * n * M2 + k2;
    const float* __restrict__ srow =
        PAD ? static_cast<const float*>(jb.S) + (long long)k0 * (n + 1) * (n2 + 1) + (ok ? min(k2, M2 - k2) : 0)
            : nullptr;
    stepA_fwd<P, V, PAD>(
        u,
        [&](int t, int r) {
          const int p = t + R2 * r;
          return (p < n && ok) ? col[(long long)p * M2] : czero<V>();
        },
        [&](int q, int t, V v) { sm[(q * R2 + t) * W + l] = v; });
    __syncthreads();
    MidSpec<P> sp;
    if constexpr (PAD) mid_load<P>(sp, srow, u, ok, n2 + 1);
    V b[R2];
#pragma unroll
    for (int t = 0; t < R2; ++t) b[t] = sm[(u * R2 + t) * W + l];
    rfft<R2, true>(b);
    // b[s] = transform at k1 = u + R1 s: multiply by the spectrum (real, even)
    mid_multiply<P, MODE>(b, sp, u, jb, k0, k2, M2, ok);
    // the locations this thread read are the ones it writes: no barrier needed
    stepB_inv<P, V>(u, b, [&](int q, int t, V v) { sm[(q * R2 + t) * W + l] = v; });
    __syncthreads();
    stepA_inv<P, V, PAD>(
        u, [&](int q, int t) { return sm[(q * R2 + t) * W + l]; },
        [&](int t, int r, V v) {
          const int p = t + R2 * r;
          if (p < n && ok) col[(long long)p * M2] = v;
        });
    __syncthreads();
  }
}

// ----------------------------------------------- pass 3, prefetching form --
// Async copy of 8 bytes global -> shared; src_bytes = 0 writes zeros instead
// (pruned or out-of-range elements).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The middle pass with step A's inputs of the next tile copied asynchronously
// into a staging area while the current tile computes.  Each thread stages
// and later reads only its own elements (t = u + T i, r < RA), so a thread's
// own cp.async.wait orders the copy before its reads.
template <class P> struct Stage2 {
  static constexpr int RA = (P::R1 + 1) / 2;  // loads per step-A sub-transform (the rest is zero padding)
  static constexpr int SLOTS = P::PA * RA;
  static constexpr int BYTES = SLOTS * P::T * Geo2<P>::W * 8;
};

// SHARED: every job of the launch has the same spectrum (densities of one
// plan).  A CTA then takes a column tile for all jobs in turn and loads the
// tile's spectrum values once (one spectrum read per tile, not per job).
template <class P, int MODE = kMulSpectrum, bool SHARED = false>
__global__ void __launch_bounds__(Geo2<P>::NT, Geo2<P>::MINB_MID) k2p_col_mid(const Jobs jobs, int M2, int planes) {
  using V = float2;
  constexpr int M = P::M, n = M / 2, W = Geo2<P>::W, R1 = P::R1, R2 = P::R2, T = P::T;
  constexpr int RA = Stage2<P>::RA;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  V* stg = sm + M * W;  // staging: [slot][u][l]
  const int l = threadIdx.x % W, u = mid_u<P>(threadIdx.x);
  const int tiles_per_plane = (M2 + W - 1) / W;
  const long long tpj = (long long)tiles_per_plane * planes;
  const long long K = jobs.count;
  const long long total = tpj * K;
  const int n2 = M2 / 2;
  // work item -> (job, tile of the job); SHARED orders the jobs innermost;
  // kMidReverse walks the items from the last
  auto ph = [&](long long tile) -> long long { return kMidReverse ? total - 1 - tile : tile; };
  auto job_of = [&](long long tile) -> int { return (int)(SHARED ? ph(tile) % K : ph(tile) / tpj); };
  auto lt_of = [&](long long tile) -> int { return (int)(SHARED ? ph(tile) / K : ph(tile) % tpj); };
  auto next_of = [&](long long tile) -> long long {
    if constexpr (SHARED) return tile % K + 1 < K ? tile + 1 : (tile / K + gridDim.x) * K;
    else return tile + gridDim.x;
  };
  const long long first = SHARED ? (long long)blockIdx.x * K : (long long)blockIdx.x;
  auto issue = [&](long long tile) {
    const Job& jb = jobs.j[job_of(tile)];
    const int lt = lt_of(tile);
    const int k0 = lt / tiles_per_plane;
    const int k2 = (lt % tiles_per_plane) * W + l;
    const bool ok = k2 < M2;
    const V* col = static_cast<const V*>(jb.out) + (long long)k0 * n * M2 + (ok ? k2 : 0);
#pragma unroll
    for (int i = 0; i < P::PA; ++i) {
#pragma unroll
      for (int r = 0; r < RA; ++r) {
        const int t = u + T * i;
        const int p = t + R2 * r;
        const bool live = ok && t < R2 && p < n;
        cp_async8(&stg[((i * RA + r) * T + u) * W + l], live ? col + (long long)p * M2 : col, live ? 8 : 0);
      }
    }
    cp_async_commit();
  };
  if (first < total) issue(first);
  MidSpec<P> sp;
  for (long long tile = first; tile < total; tile = next_of(tile)) {
    const int job = job_of(tile);
    const Job& jb = jobs.j[job];
    const int lt = lt_of(tile);
    const int k0 = lt / tiles_per_plane;
    const int k2 = (lt % tiles_per_plane) * W + l;
    const bool ok = k2 < M2;
    V* __restrict__ col = static_cast<V*>(jb.out) + (long long)k0 * n * M2 + k2;
    const float* __restrict__ srow =
        static_cast<const float*>(jb.S) + (long long)k0 * (n + 1) * (n2 + 1) + (ok ? min(k2, M2 - k2) : 0);
    cp_async_wait_all();
    stepA_fwd<P, V, true>(
        u,
        [&](int t, int r) {
          const int i = (t - u) / T;
          return r < RA ? stg[((i * RA + r) * T + u) * W + l] : czero<V>();
        },
        [&](int q, int t, V v) { sm[(q * R2 + t) * W + l] = v; });
    // this thread's staged elements are consumed: fetch the next tile's
    if (next_of(tile) < total) issue(next_of(tile));
    __syncthreads();
    // SHARED: the first job of the group this CTA takes in turn loads the tile's spectrum
    if (!SHARED || tile % K == 0) mid_load<P>(sp, srow, u, ok, n2 + 1);
    V b[R2];
#pragma unroll
    for (int t = 0; t < R2; ++t) b[t] = sm[(u * R2 + t) * W + l];
    rfft<R2, true>(b);
    mid_multiply<P, MODE>(b, sp, u, jb, k0, k2, M2, ok);
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
  cp_async_wait_all();
}

// ------------------------------------------ row passes, prefetching form --
// WR rows per CTA, lanes on the R1 threads of a row.  Step A (forward) or
// step B (inverse) inputs of the next tile are copied asynchronously into a
// per-thread staging area while the current tile computes.
template <class P, int WR> struct RowGeo {
  static constexpr int NT = WR * P::T;
  static constexpr int PITCH = P::R1 * (P::R2 + 1);
  static constexpr int RA = (P::R1 + 1) / 2;
  static constexpr int XCH = WR * PITCH * 8;                      // exchange tile
  static constexpr int STG_FWD = P::PA * RA * P::T * WR * 8;      // step-A inputs
  static constexpr int STG_INV = P::R2 * P::T * WR * 8;           // step-B inputs
  static constexpr int SM_FWD = XCH + STG_FWD;
  static constexpr int SM_INV = XCH + STG_INV;
};

template <class P, int WR>
__global__ void __launch_bounds__(RowGeo<P, WR>::NT) k2p_row_fwd(const Jobs jobs, long long rows) {
  using V = float2;
  using G = RowGeo<P, WR>;
  constexpr int M = P::M, n = M / 2, R1 = P::R1, R2 = P::R2, T = P::T, RA = G::RA;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  V* stg = sm + WR * G::PITCH;  // [slot][l][u]
  const int u = threadIdx.x % T, l = threadIdx.x / T;
  V* line = sm + l * G::PITCH;
  const long long tpj = (rows + WR - 1) / WR;
  const long long total = tpj * jobs.count;
  auto issue = [&](long long tile) {
    const Job& jb = jobs.j[tile / tpj];
    const long long row = (tile % tpj) * WR + l;
    const bool ok = row < rows;
    const V* x = static_cast<const V*>(jb.in) + (ok ? row : 0) * n;
#pragma unroll
    for (int i = 0; i < P::PA; ++i) {
#pragma unroll
      for (int r = 0; r < RA; ++r) {
        const int t = u + T * i;
        const int p = t + R2 * r;
        const bool live = ok && t < R2 && p < n;
        cp_async8(&stg[((i * RA + r) * WR + l) * T + u], live ? x + p : x, live ? 8 : 0);
      }
    }
    cp_async_commit();
  };
  if (blockIdx.x < total) issue(blockIdx.x);
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const Job& jb = jobs.j[tile / tpj];
    const long long row = (tile % tpj) * WR + l;
    const bool ok = row < rows;
    V* __restrict__ y = static_cast<V*>(jb.out) + row * M;
    cp_async_wait_all();
    stepA_fwd<P, V, true>(
        u,
        [&](int t, int r) {
          const int i = (t - u) / T;
          return r < RA ? stg[((i * RA + r) * WR + l) * T + u] : czero<V>();
        },
        [&](int q, int t, V v) { line[q * (R2 + 1) + t] = v; });
    if (tile + gridDim.x < total) issue(tile + gridDim.x);
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
  cp_async_wait_all();
}

template <class P, int WR>
__global__ void __launch_bounds__(RowGeo<P, WR>::NT) k2p_row_inv(const Jobs jobs, long long rows) {
  using V = float2;
  using G = RowGeo<P, WR>;
  constexpr int M = P::M, n = M / 2, R1 = P::R1, R2 = P::R2, T = P::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  V* stg = sm + WR * G::PITCH;  // [s][l][u]
  const int u = threadIdx.x % T, l = threadIdx.x / T;
  V* line = sm + l * G::PITCH;
  const long long tpj = (rows + WR - 1) / WR;
  const long long total = tpj * jobs.count;
  auto issue = [&](long long tile) {
    const Job& jb = jobs.j[tile / tpj];
    const long long row = (tile % tpj) * WR + l;
    const bool ok = row < rows;
    const V* y = static_cast<const V*>(jb.in) + (ok ? row : 0) * M;
#pragma unroll
    for (int s = 0; s < R2; ++s) cp_async8(&stg[(s * WR + l) * T + u], y + u + R1 * s, ok ? 8 : 0);
    cp_async_commit();
  };
  if (blockIdx.x < total) issue(blockIdx.x);
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const Job& jb = jobs.j[tile / tpj];
    const long long row = (tile % tpj) * WR + l;
    const bool ok = row < rows;
    V* __restrict__ x = static_cast<V*>(jb.out) + row * n;
    cp_async_wait_all();
    V b[R2];
#pragma unroll
    for (int s = 0; s < R2; ++s) b[s] = stg[(s * WR + l) * T + u];
    if (tile + gridDim.x < total) issue(tile + gridDim.x);
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
  cp_async_wait_all();
}

// ---------------------------------------------------------------- pass 4 --
template <class P>
__global__ void __launch_bounds__(Geo2<P>::NT) k2_row_inv(const Jobs jobs, long long rows) {
  using V = float2;
  constexpr int M = P::M, n = M / 2, W = Geo2<P>::W, R1 = P::R1, R2 = P::R2, PITCH = Geo2<P>::PITCH;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int u = threadIdx.x % P::T, l = threadIdx.x / P::T;
  V* line = sm + l * PITCH;
  const long long tpj = (rows + W - 1) / W;
  for (long long tile = blockIdx.x; tile < tpj * jobs.count; tile += gridDim.x) {
    const Job& jb = jobs.j[tile / tpj];
    const long long row = (tile % tpj) * W + l;
    const bool ok = row < rows;
    const V* __restrict__ y = static_cast<const V*>(jb.in) + row * M;
    V* __restrict__ x = static_cast<V*>(jb.out) + row * n;
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
}

// ---------------------------------------------------------------- pass 5 --
// EPI: phi + beta * rho (rho = jb.aux, beta = the DDI block's kDdiBeta), the
// DDI grid reading's local term.  The rho values this thread will add are
// loaded at the start of the tile, before any store (phi may be rho).
template <class P, bool EPI = false, bool PAD = true>
__global__ void __launch_bounds__(Geo2<P>::NT) k2_c2r_ax0(const Jobs jobs, long long C) {
  using V = float2;
  constexpr int M = P::M, n = M / 2, NV = PAD ? M / 2 : M, W = Geo2<P>::W, R1 = P::R1, R2 = P::R2;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int l = threadIdx.x % W, u = threadIdx.x / W;
  const long long tpj = (C + 2 * W - 1) / (2 * W);
  for (long long tile = blockIdx.x; tile < tpj * jobs.count; tile += gridDim.x) {
    const Job& jb = jobs.j[tile / tpj];
    const V* __restrict__ X = static_cast<const V*>(jb.in);
    float* __restrict__ phi = static_cast<float*>(jb.out);
    const long long c = (tile % tpj) * (2 * W) + 2 * l;
    const bool ok = c < C;
    constexpr int RH = PAD && R1 % 2 == 0 ? R1 / 2 : R1;  // outputs per sub-transform (step A keeps p < NV)
    V rr[EPI ? P::PA : 1][EPI ? RH : 1];
    if constexpr (EPI) {
      const float* rho = static_cast<const float*>(jb.aux);
#pragma unroll
      for (int i = 0; i < P::PA; ++i) {
#pragma unroll
        for (int r = 0; r < RH; ++r) {
          const int t = u + P::T * i, p = t + R2 * r;
          rr[i][r] = (ok && t < R2 && p < NV) ? *reinterpret_cast<const V*>(rho + (long long)p * C + c) : czero<V>();
        }
      }
    }
    // Z[k] = A[k] + i B[k] with A, B Hermitian: rebuild k > n from M - k.
    V b[R2];
#pragma unroll
    for (int s = 0; s < R2; ++s) {
      const int k = u + R1 * s;
      V z = czero<V>();
      if (ok) {
        const bool lo = k <= n;
        const long long kk = lo ? k : M - k;
        // columns c and c + 1 are adjacent (c even, C even): one 16-byte load
        const float4 ab = *reinterpret_cast<const float4*>(X + kk * C + c);
        z = lo ? mk(ab.x - ab.w, ab.y + ab.z) : mk(ab.x + ab.w, ab.z - ab.y);
      }
      b[s] = z;
    }
    stepB_inv<P, V>(u, b, [&](int q, int t, V v) { sm[(q * R2 + t) * W + l] = v; });
    __syncthreads();
    stepA_inv<P, V, PAD>(
        u, [&](int q, int t) { return sm[(q * R2 + t) * W + l]; },
        [&](int t, int r, V v) {
          const int p = t + R2 * r;
          if (p < NV && ok) {
            if constexpr (EPI) {
              store_pair_axpy<V>(phi + (long long)p * C + c, v, ddi_beta<float>(jb.par), rr[(t - u) / P::T][r]);
            } else {
              *reinterpret_cast<V*>(phi + (long long)p * C + c) = v;
            }
          }
        });
    __syncthreads();
  }
}

}  // namespace fsa
