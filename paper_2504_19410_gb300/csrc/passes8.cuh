// Eighth-generation FP32 middle pass: generation 2's two-step register
// transform with each column tile's inputs staged by ONE tiled bulk tensor
// copy (TMA, cp.async.bulk.tensor.2d) per tile.
//
// A middle-pass tile is W = 16 adjacent columns k2 of one axis-0 plane k0,
// over its n1 rows (Y[k0][0..n1)[k2..k2+16): n1 rows of 128 bytes, M2 x 8
// bytes apart).  Generation 2 loads them straight from HBM at the start of
// the tile (the load latency shows as long-scoreboard stalls); generation 3
// stages them with per-thread cp.async copies (extra instructions, and bank
// conflicts in its staging layout).  Here thread 0 issues one 2-D tensor copy
// of the whole n1 x 16 box into shared memory, laid out [row][column] as the
// plain loads would read it, with completion counted in bytes on an mbarrier;
// the copy of the next tile is issued as soon as every thread has taken the
// current one out of the staging buffer, and runs under the rest of the
// current tile's work.  The arithmetic is generation 2's, so the results are
// bit-equal to it.
//
// The R2C and C2R passes along axis 0 are staged the same way (k8_r2c_ax0,
// k8_c2r_ax0 below).
//
// The copies need a tensor map per solve of the launch (host-encoded per
// launch, passed in a __grid_constant__ parameter: NJ maps, NJ = 1 for a
// single solve or kMaxJobs for a launch of several).  Every wait on the
// mbarrier is bounded (kWaitLimitCycles); a CTA whose wait gives up ORs
// kWaitTimeout into jobs.fault, waits (bounded) for its copy in flight and
// returns, the decision taken CTA-wide at the barrier that ends step A.
#pragma once
#include <cuda.h>

#include "mbar.cuh"
#include "passes2.cuh"

namespace fsa {

// 2-D tiled copy global -> shared of the box at element coordinates (x, y)
// of the tensor map; x * 8 bytes is a multiple of 16 (x = 16 c).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// The tensor maps of a launch's solves (128 bytes each, 64-byte aligned).
template <int NJ> struct TmapSet {
  CUtensorMap m[NJ];
};

// Shared memory: the exchange tile (M x W complex), the staged input box
// (n1 = M/2 rows x W columns), the mbarrier.
template <class P> struct Geo8 {
  static constexpr int W = Geo2<P>::W;
  static constexpr int NT = Geo2<P>::NT;
  static constexpr int XCH = P::M * W * 8;
  static constexpr int STG = (P::M / 2) * W * 8;
  static constexpr int BAR = XCH + STG;
  static constexpr int SMEM = BAR + 16;
  static_assert(W == 16 && XCH % 16 == 0 && STG % 16 == 0, "box of 16 columns, 16-byte aligned staging");
};

// ymap.m[j]: Y of solve j as a 2-D tensor of 8-byte elements, dims
// {M2, planes * n1}, box {16, n1}.  SHARED: every solve of the launch has the
// same spectrum (densities of one plan); a CTA then takes one column tile for
// all solves in turn and loads the tile's spectrum values once.
template <class P, int NJ, bool SHARED = false>
__global__ void __launch_bounds__(Geo2<P>::NT, Geo2<P>::MINB_MID)
    k8_col_mid(const Jobs jobs, int M2, int planes, const __grid_constant__ TmapSet<NJ> ymap) {
  using V = float2;
  using G = Geo8<P>;
  constexpr int M = P::M, n = M / 2, W = G::W, R2 = P::R2;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const V* stg = reinterpret_cast<const V*>(smraw + G::XCH);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smraw + G::BAR);
  const int l = threadIdx.x % W, u = mid_u<P>(threadIdx.x);
  const int tpp = M2 / W;  // column tiles per plane
  const long long tpj = (long long)tpp * planes;  // tiles per solve
  const long long K = jobs.count;
  const long long total = tpj * K;
  const int n2 = M2 / 2;
  // work item -> (solve, tile of the solve), walked from the last item to
  // the first; SHARED orders the solves innermost and a CTA takes the K
  // items of one tile in a row
  auto phys = [&](long long it) -> long long { return kMidReverse ? total - 1 - it : it; };
  auto job_of = [&](long long it) -> long long { return SHARED ? phys(it) % K : phys(it) / tpj; };
  auto lt_of = [&](long long it) -> long long { return SHARED ? phys(it) / K : phys(it) % tpj; };
  auto next_of = [&](long long it) -> long long {
    if constexpr (SHARED) return it % K + 1 < K ? it + 1 : (it / K + gridDim.x) * K;
    else return it + gridDim.x;
  };
  const long long first = SHARED ? (long long)blockIdx.x * K : (long long)blockIdx.x;
  auto issue = [&](long long it) {  // thread 0
    const long long lt = lt_of(it);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, (unsigned)G::STG);
    tma_load_2d(smraw + G::XCH, &ymap.m[job_of(it)], (int)(lt % tpp) * W, (int)(lt / tpp) * n, bar);
  };
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && first < total) issue(first);
  MidSpec<P> sp;
  int k = 0;
  for (long long it = first; it < total; it = next_of(it), ++k) {
    const long long lt = lt_of(it);
    const Job& jb = jobs.j[job_of(it)];
    const int k0 = (int)(lt / tpp);
    const int k2 = (int)(lt % tpp) * W + l;
    V* __restrict__ col = static_cast<V*>(jb.out) + (long long)k0 * n * M2 + k2;
    const float* __restrict__ srow =
        static_cast<const float*>(jb.S) + (long long)k0 * (n + 1) * (n2 + 1) + min(k2, M2 - k2);
    const bool late = !mbar_wait(bar, k & 1);
    stepA_fwd<P, V, true>(
        u,
        [&](int t, int r) {
          const int p = t + R2 * r;
          return p < n ? stg[p * W + l] : czero<V>();
        },
        [&](int q, int t, V v) { sm[(q * R2 + t) * W + l] = v; });
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0) {
        if (jobs.fault) atomicOr(jobs.fault, kWaitTimeout);
        mbar_wait(bar, k & 1);  // the copy still in flight
      }
      __syncthreads();
      return;
    }
    // every thread has taken the tile out of the staging buffer: the next one
    if (threadIdx.x == 0 && next_of(it) < total) issue(next_of(it));
    // SHARED: the first solve of the tile this CTA takes in turn loads the spectrum
    if (!SHARED || it % K == 0) mid_load<P>(sp, srow, u, true, n2 + 1);
    V b[R2];
#pragma unroll
    for (int t = 0; t < R2; ++t) b[t] = sm[(u * R2 + t) * W + l];
    rfft<R2, true>(b);
    mid_multiply<P, kMulSpectrum>(b, sp, u, jb, k0, k2, M2, true);
    stepB_inv<P, V>(u, b, [&](int q, int t, V v) { sm[(q * R2 + t) * W + l] = v; });
    __syncthreads();
    stepA_inv<P, V, true>(
        u, [&](int q, int t) { return sm[(q * R2 + t) * W + l]; },
        [&](int t, int r, V v) {
          const int p = t + R2 * r;
          if (p < n) col[(long long)p * M2] = v;
        });
    __syncthreads();
  }
}

// The pad + R2C pass along axis 0 (pass 1) with the same staging: a tile is
// 2W = 32 adjacent real columns c of rho over its n0 rows (rows C floats
// apart), carried as W complex lines (columns c, c + 1 as one complex
// value), staged by one 2-D tensor copy of the n0 x 32 box ([row][column],
// 128 bytes a row).  rmap.m[j]: rho of solve j as a 2-D tensor of 4-byte
// elements, dims {C, n0}, box {32, n0}; columns past C read as zero.
template <class P> struct Geo8R {
  static constexpr int W = Geo2<P>::W;
  static constexpr int NT = Geo2<P>::NT;
  static constexpr int XCH = Geo2<P>::SM_STRIDED;
  static constexpr int STG = (P::M / 2) * 2 * W * 4;
  static constexpr int BAR = XCH + STG;
  static constexpr int SMEM = BAR + 16;
  static_assert(W == 16 && XCH % 16 == 0 && STG % 16 == 0, "box of 32 real columns, 16-byte aligned staging");
};

template <class P, int NJ>
__global__ void __launch_bounds__(Geo2<P>::NT, Geo2<P>::MINB_MID)
    k8_r2c_ax0(const Jobs jobs, long long C, const __grid_constant__ TmapSet<NJ> rmap) {
  using V = float2;
  using G = Geo8R<P>;
  constexpr int M = P::M, n = M / 2, K = M / 2 + 1, W = G::W, R1 = P::R1, R2 = P::R2;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const V* stg = reinterpret_cast<const V*>(smraw + G::XCH);  // [row][W complex]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smraw + G::BAR);
  const int l = threadIdx.x % W, u = threadIdx.x / W;
  const long long tpj = (C + 2 * W - 1) / (2 * W);  // tiles per solve
  const long long total = tpj * jobs.count;
  auto issue = [&](long long tile) {  // thread 0
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, (unsigned)G::STG);
    tma_load_2d(smraw + G::XCH, &rmap.m[tile / tpj], (int)((tile % tpj) * 2 * W), 0, bar);
  };
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && blockIdx.x < total) issue(blockIdx.x);
  int k = 0;
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x, ++k) {
    V* __restrict__ X = static_cast<V*>(jobs.j[tile / tpj].out);
    const long long c = (tile % tpj) * (2 * W) + 2 * l;
    const bool ok = c < C;
    const bool late = !mbar_wait(bar, k & 1);
    stepA_fwd<P, V, true>(
        u,
        [&](int t, int r) {
          const int p = t + R2 * r;
          return p < n ? stg[p * W + l] : czero<V>();
        },
        [&](int q, int t, V v) { sm[(q * R2 + t) * W + l] = v; });
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0) {
        if (jobs.fault) atomicOr(jobs.fault, kWaitTimeout);
        mbar_wait(bar, k & 1);  // the copy still in flight
      }
      __syncthreads();
      return;
    }
    if (threadIdx.x == 0 && tile + gridDim.x < total) issue(tile + gridDim.x);
    V b[R2];
#pragma unroll
    for (int t = 0; t < R2; ++t) b[t] = sm[(u * R2 + t) * W + l];
    rfft<R2, true>(b);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < R2; ++s) sm[(u + R1 * s) * W + l] = b[s];
    __syncthreads();
    // Z = DFT(a + i b): A[k] = (Z[k] + conj Z[M-k]) / 2, B[k] = (Z[k] - conj Z[M-k]) / 2i
    for (int kk = u; kk < K; kk += P::T) {
      const V zk = sm[kk * W + l];
      const V zm = sm[((M - kk) % M) * W + l];
      if (ok) {
        *reinterpret_cast<float4*>(X + (long long)kk * C + c) =
            make_float4(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y), 0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
      }
    }
    __syncthreads();
  }
}

// The C2R pass along axis 0 + crop (pass 5) with the same staging.  Its
// tile reads all K0 = n0 + 1 rows of X (the half spectrum: rows k <= n0
// directly, k > n0 from their mirror M - k), 2 x W8 complex columns a row; at
// W = 16 the staged box and the exchange tile would take 130 KB and leave one
// CTA per SM, so this pass runs W8 = 8 complex lines (16 real columns) per
// CTA of 128 threads: a 258-row box of 128-byte rows (two copies of 129 rows,
// 33 KB; the last row lies past X and reads as zero) and a 32 KB exchange
// tile, three CTAs per SM.  xmap.m[j]: X of solve j as a 2-D tensor of
// 8-byte elements, dims {C, K0}, box {16, 129}.
template <class P> struct Geo8C {
  static constexpr int W = 8;
  static constexpr int NT = W * P::T;
  static constexpr int ROWS = 2 * ((P::M / 2 + 2) / 2);  // K0 = M/2 + 1 rows, rounded up to two equal boxes
  static constexpr int XCH = P::M * W * 8;
  static constexpr int STG = ROWS * 2 * W * 8;
  static constexpr int BAR = XCH + STG;
  static constexpr int SMEM = BAR + 16;
  static_assert(ROWS / 2 <= 256 && XCH % 16 == 0 && STG % 16 == 0, "two boxes of at most 256 rows");
};

template <class P, int NJ>
__global__ void __launch_bounds__(Geo8C<P>::NT, 3)
    k8_c2r_ax0(const Jobs jobs, long long C, const __grid_constant__ TmapSet<NJ> xmap) {
  using V = float2;
  using G = Geo8C<P>;
  constexpr int M = P::M, n = M / 2, W = G::W, R1 = P::R1, R2 = P::R2;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const float4* stg = reinterpret_cast<const float4*>(smraw + G::XCH);  // [row][W column pairs]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smraw + G::BAR);
  const int l = threadIdx.x % W, u = threadIdx.x / W;
  const long long tpj = (C + 2 * W - 1) / (2 * W);  // tiles per solve
  const long long total = tpj * jobs.count;
  auto issue = [&](long long tile) {  // thread 0
    const CUtensorMap* map = &xmap.m[tile / tpj];
    const int x = (int)((tile % tpj) * 2 * W);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, (unsigned)G::STG);
    tma_load_2d(smraw + G::XCH, map, x, 0, bar);
    tma_load_2d(smraw + G::XCH + G::STG / 2, map, x, G::ROWS / 2, bar);
  };
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && blockIdx.x < total) issue(blockIdx.x);
  int it = 0;
  for (long long tile = blockIdx.x; tile < total; tile += gridDim.x, ++it) {
    float* __restrict__ phi = static_cast<float*>(jobs.j[tile / tpj].out);
    const long long c = (tile % tpj) * (2 * W) + 2 * l;
    const bool ok = c < C;
    const bool late = !mbar_wait(bar, it & 1);
    // Z[k] = A[k] + i B[k] with A, B Hermitian: rebuild k > n from M - k
    V b[R2];
#pragma unroll
    for (int s = 0; s < R2; ++s) {
      const int k = u + R1 * s;
      const bool lo = k <= n;
      const float4 ab = stg[(lo ? k : M - k) * W + l];
      b[s] = lo ? mk(ab.x - ab.w, ab.y + ab.z) : mk(ab.x + ab.w, ab.z - ab.y);
    }
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0) {
        if (jobs.fault) atomicOr(jobs.fault, kWaitTimeout);
        mbar_wait(bar, it & 1);  // the copies still in flight
      }
      __syncthreads();
      return;
    }
    // every thread holds its inputs: the next tile's copies run under this one
    if (threadIdx.x == 0 && tile + gridDim.x < total) issue(tile + gridDim.x);
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
}

}  // namespace fsa
