// The five apply passes of the pruned zero-padded 3-D convolution and the
// DCT-I pass of tensor generation, as templates over the complex type
// (float2 / double2), the transform plan (length M = 2n) and the tile shape
// (W lines per CTA, T threads per line).
//
// Data flow of one solve (Sec. 2.3: FFT over the doubled grid, pointwise
// multiply by the spectrum of T, inverse FFT, keep the first n_j entries):
//
//   rho [n0][n1][n2] real
//     -- r2c_ax0 : pad axis 0 to M0, real FFT (two real lines per complex
//                  line), keep k0 in [0, n0]                 -> X [n0+1][n1][n2]
//     -- row_fwd : pad axis 2 to M2, FFT                        -> Y [n0+1][n1][M2]
//     -- col_mid : pad axis 1 to M1, FFT, multiply by the
//                  spectrum, inverse FFT, keep n1  (in place)   -> Y
//     -- row_inv : inverse FFT axis 2, keep n2                  -> X
//     -- c2r_ax0 : inverse real FFT axis 0, keep n0             -> phi [n0][n1][n2]
//
// Zero inputs of the padded half are never read (pruned loads), discarded
// outputs are never written (pruned stores).  The spectrum is stored as the
// octant S[p0][p1][p2], p_j in [0, n_j]; the full even spectrum is
// S[min(k, M-k)] per axis.  The inverse normalisation is folded into S.
//
// Layouts in shared memory.  Strided passes (axes 0 and 1) keep a tile of W
// lines as sm[p * W + l] and map lanes to lines, so every global access of a
// warp touches consecutive addresses of the contiguous axis.  Row passes
// (axis 2) copy W rows in with coalesced loads to sm[l * (M+1) + p] (odd
// pitch: lanes on different rows hit different banks), transform them with
// lanes mapped to rows, and copy them out coalesced.
#pragma once
#include "ddi.cuh"
#include "fft_core.cuh"

namespace fsa {

template <typename V> struct TileW { static constexpr int W = 16; };
template <> struct TileW<double2> { static constexpr int W = 8; };
template <> struct TileW<cdw> { static constexpr int W = 4; };

// Resident CTAs per SM the compiler should allow for: double-word passes are
// bound by the FP32 pipes; they run 4-line tiles (256 threads for length
// 512) four to an SM (at most 64 registers), so a barrier holds fewer warps
// (R2C 0.218 against 0.255 ms, C2R 0.204 against 0.230 ms at 256^3 with
// 8-line tiles two to an SM; the row passes the same).
template <typename V> struct MinB { static constexpr int value = 1; };
template <> struct MinB<cdw> { static constexpr int value = 4; };

// The middle pass keeps a whole line's forward transform, multiply and
// inverse in one CTA; for double-word values it takes half-width tiles so
// that two CTAs (each up to 128 registers a thread) share an SM and one's
// barriers and loads overlap the other's arithmetic.
template <typename V> struct MidW { static constexpr int W = TileW<V>::W; };
template <> struct MidW<cdw> { static constexpr int W = 4; };
template <typename V, int NT> constexpr int minb_mid() { return (std::is_same<V, cdw>::value && NT <= 256) ? 2 : 1; }

// Threads per line: one butterfly of the largest radix per thread, capped so
// that a CTA has at most 512 threads.
template <class P, int W> constexpr int threads_per_line() {
  int t = P::M / P::rmax();
  int cap = 512 / W;
  if (t > cap) t = cap;
  return t < 1 ? 1 : t;
}

template <class P, typename V, int W> constexpr int smem_strided() { return P::M * W * (int)sizeof(V); }
template <class P, typename V, int W> constexpr int smem_rows() { return W * (P::M + 1) * (int)sizeof(V); }

// ---------------------------------------------------------------- pass 1 --
// Every kernel walks the tiles of all jobs of its launch with a grid-strided
// loop (a persistent grid of a few CTAs per SM).
// PAD = false: the unpadded transform of length M over all M inputs (the DDI
// grid reading's derivative, Sec. 5 Example 4); the same K = M/2 + 1 outputs.
template <typename V, class P, int W, int T, bool PAD = true>
__global__ void __launch_bounds__(W * T, MinB<V>::value) k_r2c_ax0(const Jobs jobs, long long C) {
  using R = typename RealOf<V>::T;
  constexpr int M = P::M, NV = PAD ? M / 2 : M, K = M / 2 + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int l = threadIdx.x % W, t = threadIdx.x / W;
  const long long tpj = (C + 2 * W - 1) / (2 * W);
  for (long long tile = blockIdx.x; tile < tpj * jobs.count; tile += gridDim.x) {
  const Job& jb = jobs.j[tile / tpj];
  const typename Io<V>::T* __restrict__ rho = static_cast<const typename Io<V>::T*>(jb.in);
  V* __restrict__ X = static_cast<V*>(jb.out);
  const long long c = (tile % tpj) * (2 * W) + 2 * l;  // first of the two real columns
  const bool ok = c < C;
  SLine<V, W> sl{sm + l};
  auto first = [&](int p) -> V {
    return (p < NV && ok) ? load_pair<V>(rho + (long long)p * C + c) : czero<V>();
  };
  auto last = [&](int p, V v) { sl.put(p, v); };
  fft_line<P, true, T, V, PAD, false>(t, first, last, sl);
  // Z = DFT(a + i b): A[k] = (Z[k] + conj Z[M-k]) / 2, B[k] = (Z[k] - conj Z[M-k]) / 2i
  for (int k = t; k < K; k += T) {
    const V zk = sm[k * W + l];
    const V zm = sm[((M - k) % M) * W + l];
    const V a = mk(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
    const V b = mk(R(0.5) * (zk.y + zm.y), R(0.5) * (zm.x - zk.x));
    if (ok) {
      X[(long long)k * C + c] = canon(a);
      X[(long long)k * C + c + 1] = canon(b);
    }
  }
  __syncthreads();
  }
}

// ---------------------------------------------------------------- pass 2 --
template <typename V, class P, int W, int T, bool PAD = true>
__global__ void __launch_bounds__(W * T, MinB<V>::value) k_row_fwd(const Jobs jobs, long long rows) {
  constexpr int M = P::M, n = PAD ? M / 2 : M, PITCH = M + 1, NT = W * T;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const long long tpj = (rows + W - 1) / W;
  for (long long tile = blockIdx.x; tile < tpj * jobs.count; tile += gridDim.x) {
  const Job& jb = jobs.j[tile / tpj];
  const V* __restrict__ X = static_cast<const V*>(jb.in);
  V* __restrict__ Y = static_cast<V*>(jb.out);
  const long long row0 = (tile % tpj) * W;
  for (int i = threadIdx.x; i < W * n; i += NT) {
    const int l = i / n, p = i - l * n;
    const long long row = row0 + l;
    sm[l * PITCH + p] = row < rows ? X[row * n + p] : czero<V>();
  }
  __syncthreads();
  const int l = threadIdx.x % W, t = threadIdx.x / W;
  SLine<V, 1> sl{sm + l * PITCH};
  auto first = [&](int p) -> V { return p < n ? sl.get(p) : czero<V>(); };
  auto last = [&](int p, V v) { sl.put(p, v); };
  fft_line<P, true, T, V, PAD, false>(t, first, last, sl);
  for (int i = threadIdx.x; i < W * M; i += NT) {
    const int l2 = i / M, p = i - l2 * M;
    const long long row = row0 + l2;
    if (row < rows) Y[row * M + p] = canon(sm[l2 * PITCH + p]);
  }
  __syncthreads();
  }
}

// ---------------------------------------------------------------- pass 3 --
// MODE (ddi.cuh): kMulSpectrum multiplies by the stored spectrum; the DDI
// modes by the multiplier of jb.par, kMulDdiGrid on the unpadded grid (all
// M entries of a column live, transform length M along every axis).
template <typename V, class P, int W, int T, int MODE = kMulSpectrum>
__global__ void __launch_bounds__(W * T, minb_mid<V, W * T>()) k_col_mid(const Jobs jobs, int M2, int planes) {
  using R = typename RealOf<V>::T;
  constexpr bool PAD = MODE != kMulDdiGrid;
  constexpr int M = P::M, n = PAD ? M / 2 : M;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int l = threadIdx.x % W, t = threadIdx.x / W;
  const int tiles_per_plane = (M2 + W - 1) / W;
  const long long tpj = (long long)tiles_per_plane * planes;
  for (long long tile = blockIdx.x; tile < tpj * jobs.count; tile += gridDim.x) {
  const Job& jb = jobs.j[tile / tpj];
  V* __restrict__ Y = static_cast<V*>(jb.out);
  const typename Io<V>::S* __restrict__ S = static_cast<const typename Io<V>::S*>(jb.S);
  const int lt = (int)(tile % tpj);
  const int k0 = lt / tiles_per_plane;
  const int k2 = (lt % tiles_per_plane) * W + l;
  const bool ok = k2 < M2;
  const int n2 = M2 / 2;
  const int p2 = ok ? min(k2, M2 - k2) : 0;
  V* col = Y + (long long)k0 * n * M2 + k2;
  const typename Io<V>::S* srow = PAD ? S + (long long)k0 * (n + 1) * (n2 + 1) + p2 : S;
  SLine<V, W> sl{sm + l};
  auto first = [&](int p) -> V { return (p < n && ok) ? col[(long long)p * M2] : czero<V>(); };
  auto to_sm = [&](int p, V v) { sl.put(p, v); };
  fft_line<P, true, T, V, PAD, false>(t, first, to_sm, sl);
  // the line's DDI coefficients, loaded here rather than held across the
  // forward transform (registers)
  DdiLine<V> ddi;
  if constexpr (MODE != kMulSpectrum) ddi.init(jb.par, k0, ok ? k2 : 0, M2);
  auto mul = [&](int p) -> V {
    R s = R(0);
    if constexpr (MODE != kMulDdiGrid) s = ok ? load_spec<V>(srow + (long long)min(p, M - p) * (n2 + 1)) : R(0);
    if constexpr (MODE != kMulSpectrum) s = ok ? ddi.template value<MODE>(s, p, M) : R(0);
    return cscale(sl.get(p), s);
  };
  auto last = [&](int p, V v) {
    if (p < n && ok) col[(long long)p * M2] = canon(v);
  };
  fft_line<P, false, T, V, false, PAD>(t, mul, last, sl);
  }
}

// ------------------------------------------------- middle pass, d = 2 --
// The 2-D path's middle pass (Sec. 2.3 with d = 2): after the R2C pass along
// axis 0, each row k0 of X (n1 = M/2 complex values, contiguous) is padded to
// M, transformed, multiplied by the spectrum S[k0][min(k1, M - k1)] (real,
// even; row stride n1 + 1), transformed back and cropped to n1 values, in
// place.  W rows per CTA in an odd-pitch shared tile, as the row passes.
template <typename V, class P, int W, int T>
__global__ void __launch_bounds__(W * T, MinB<V>::value) k_row_mid(const Jobs jobs, long long rows) {
  using R = typename RealOf<V>::T;
  constexpr int M = P::M, n = M / 2, PITCH = M + 1, NT = W * T;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const long long tpj = (rows + W - 1) / W;
  for (long long tile = blockIdx.x; tile < tpj * jobs.count; tile += gridDim.x) {
  const Job& jb = jobs.j[tile / tpj];
  V* __restrict__ X = static_cast<V*>(jb.out);
  const typename Io<V>::S* __restrict__ S = static_cast<const typename Io<V>::S*>(jb.S);
  const long long row0 = (tile % tpj) * W;
  for (int i = threadIdx.x; i < W * n; i += NT) {
    const int l = i / n, p = i - l * n;
    const long long row = row0 + l;
    sm[l * PITCH + p] = row < rows ? X[row * n + p] : czero<V>();
  }
  __syncthreads();
  const int l = threadIdx.x % W, t = threadIdx.x / W;
  const long long row = row0 + l;
  const bool ok = row < rows;
  const typename Io<V>::S* srow = S + (ok ? row : 0) * (n + 1);
  SLine<V, 1> sl{sm + l * PITCH};
  auto first = [&](int p) -> V { return p < n ? sl.get(p) : czero<V>(); };
  auto to_sm = [&](int p, V v) { sl.put(p, v); };
  fft_line<P, true, T, V, true, false>(t, first, to_sm, sl);
  auto mul = [&](int p) -> V {
    const R sv = ok ? load_spec<V>(srow + min(p, M - p)) : R(0);
    return cscale(sl.get(p), sv);
  };
  fft_line<P, false, T, V, false, true>(t, mul, to_sm, sl);
  for (int i = threadIdx.x; i < W * n; i += NT) {
    const int l2 = i / n, p = i - l2 * n;
    const long long r2 = row0 + l2;
    if (r2 < rows) X[r2 * n + p] = canon(sm[l2 * PITCH + p]);
  }
  __syncthreads();
  }
}

// ---------------------------------------------------------------- pass 4 --
template <typename V, class P, int W, int T, bool PAD = true>
__global__ void __launch_bounds__(W * T, MinB<V>::value) k_row_inv(const Jobs jobs, long long rows) {
  constexpr int M = P::M, n = PAD ? M / 2 : M, PITCH = M + 1, NT = W * T;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const long long tpj = (rows + W - 1) / W;
  for (long long tile = blockIdx.x; tile < tpj * jobs.count; tile += gridDim.x) {
  const Job& jb = jobs.j[tile / tpj];
  const V* __restrict__ Y = static_cast<const V*>(jb.in);
  V* __restrict__ X = static_cast<V*>(jb.out);
  const long long row0 = (tile % tpj) * W;
  for (int i = threadIdx.x; i < W * M; i += NT) {
    const int l = i / M, p = i - l * M;
    const long long row = row0 + l;
    sm[l * PITCH + p] = row < rows ? Y[row * M + p] : czero<V>();
  }
  __syncthreads();
  const int l = threadIdx.x % W, t = threadIdx.x / W;
  SLine<V, 1> sl{sm + l * PITCH};
  auto first = [&](int p) -> V { return sl.get(p); };
  auto last = [&](int p, V v) { sl.put(p, v); };
  fft_line<P, false, T, V, false, PAD>(t, first, last, sl);
  for (int i = threadIdx.x; i < W * n; i += NT) {
    const int l2 = i / n, p = i - l2 * n;
    const long long row = row0 + l2;
    if (row < rows) X[row * n + p] = canon(sm[l2 * PITCH + p]);
  }
  __syncthreads();
  }
}

// ---------------------------------------------------------------- pass 5 --
// EPI: the output is phi + beta * rho with rho = jb.aux, beta = the DDI block's kDdiBeta
// (the DDI grid reading's local term).
template <typename V, class P, int W, int T, bool PAD = true, bool EPI = false>
__global__ void __launch_bounds__(W * T, MinB<V>::value) k_c2r_ax0(const Jobs jobs, long long C) {
  using R = typename RealOf<V>::T;
  constexpr int M = P::M, n = M / 2, NV = PAD ? M / 2 : M;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int l = threadIdx.x % W, t = threadIdx.x / W;
  const long long tpj = (C + 2 * W - 1) / (2 * W);
  for (long long tile = blockIdx.x; tile < tpj * jobs.count; tile += gridDim.x) {
  const Job& jb = jobs.j[tile / tpj];
  const V* __restrict__ X = static_cast<const V*>(jb.in);
  typename Io<V>::T* __restrict__ phi = static_cast<typename Io<V>::T*>(jb.out);
  const long long c = (tile % tpj) * (2 * W) + 2 * l;
  const bool ok = c < C;
  SLine<V, W> sl{sm + l};
  // Z[k] = A[k] + i B[k] with A, B Hermitian: rebuild k > n from M - k.
  auto first = [&](int k) -> V {
    if (!ok) return czero<V>();
    const bool lo = k <= n;
    const long long kk = lo ? k : M - k;
    const V a = X[kk * C + c], b = X[kk * C + c + 1];
    return lo ? mk(a.x - b.y, a.y + b.x) : mk(a.x + b.y, b.x - a.y);
  };
  if constexpr (!EPI) {
    auto last = [&](int p, V v) {
      if (p < NV && ok) store_pair<V>(phi + (long long)p * C + c, v);
    };
    fft_line<P, false, T, V, false, PAD>(t, first, last, sl);
  } else {
    // The outputs stay in shared memory; the tile's rho values are all
    // loaded before any of its stores (phi may be rho: each element is read
    // and written by the same thread), then added.
    auto to_sm = [&](int p, V v) { sl.put(p, v); };
    fft_line<P, false, T, V, false, PAD>(t, first, to_sm, sl);
    using A = typename PairOf<V>::T;
    using IoT = typename Io<V>::T;
    constexpr int NT = W * T, PER = (W * NV + NT - 1) / NT;
    const IoT* rho = static_cast<const IoT*>(jb.aux);
    const IoT beta = ddi_beta<IoT>(jb.par);
    const long long cb = (tile % tpj) * (2 * W);
    A a[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = threadIdx.x + k * NT, l2 = i % W, p = i / W;
      const long long cc = cb + 2 * l2;
      a[k] = (p < NV && cc < C) ? load_rho_pair<V>(rho + (long long)p * C + cc) : A{};
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = threadIdx.x + k * NT, l2 = i % W, p = i / W;
      const long long cc = cb + 2 * l2;
      if (p < NV && cc < C) store_pair_axpy<V>(phi + (long long)p * C + cc, sm[p * W + l2], beta, a[k]);
    }
    __syncthreads();
  }
  }
}

// ------------------------------------------------------------- DCT-I pass --
// In place on an FP64 array: for each line (n+1 values O[0..n] with element
// stride es), O[p] <- O[0] + (-1)^p O[n] + 2 sum_{j=1}^{n-1} O[j] cos(pi j p / n),
// i.e. the length-2n DFT of the even extension O[min(m, 2n-m)].  Two lines
// ride in one complex transform (their DFTs are real, so they come back as
// the real and imaginary parts).  Line L starts at (L / inner) * os + (L % inner) * is.
template <class P, int W, int T>
__global__ void __launch_bounds__(W * T) k_dct1(double* __restrict__ O, long long nlines, long long inner,
                                                long long os, long long is, long long es) {
  constexpr int M = P::M, n = M / 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  const int l = threadIdx.x % W, t = threadIdx.x / W;
  const long long q = (long long)blockIdx.x * W + l;
  const long long L0 = 2 * q, L1 = 2 * q + 1;
  const bool ok0 = L0 < nlines, ok1 = L1 < nlines;
  const long long b0 = ok0 ? (L0 / inner) * os + (L0 % inner) * is : 0;
  const long long b1 = ok1 ? (L1 / inner) * os + (L1 % inner) * is : 0;
  SLine<double2, W> sl{sm + l};
  auto first = [&](int m) -> double2 {
    const long long mm = m <= n ? m : M - m;
    return mk(ok0 ? O[b0 + mm * es] : 0.0, ok1 ? O[b1 + mm * es] : 0.0);
  };
  auto last = [&](int p, double2 v) {
    if (p <= n) {
      if (ok0) O[b0 + p * es] = v.x;
      if (ok1) O[b1 + p * es] = v.y;
    }
  };
  fft_line<P, true, T, double2>(t, first, last, sl);
}

}  // namespace fsa
