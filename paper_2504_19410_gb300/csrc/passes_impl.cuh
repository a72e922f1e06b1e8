// Host-side launchers of the apply passes for one complex type V, included
// by passes_f32.cu (V = float2) and passes_f64.cu (V = double2).
#pragma once
#include <mutex>
#include <type_traits>
#include <vector>

#include "fsa_internal.h"
#include "passes.cuh"
#include "passes2.cuh"

namespace fsa {

namespace detail {

template <typename V, int M> struct Inst {
  using P = typename PlanFor<M>::type;
  static constexpr int W = TileW<V>::W;
  static constexpr int T = threads_per_line<P, W>();
  static constexpr int NT = W * T;
  static constexpr int SM_STRIDED = smem_strided<P, V, W>();
  static constexpr int SM_ROWS = smem_rows<P, V, W>();

  static cudaError_t prepare() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f, int bytes) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    set((const void*)k_r2c_ax0<V, P, W, T>, SM_STRIDED);
    set((const void*)k_row_fwd<V, P, W, T>, SM_ROWS);
    set((const void*)k_col_mid<V, P, W, T>, SM_STRIDED);
    set((const void*)k_row_inv<V, P, W, T>, SM_ROWS);
    set((const void*)k_c2r_ax0<V, P, W, T>, SM_STRIDED);
    return e;
  }
  static Geometry geometry(PassKind k) {
    Geometry g;
    g.W = W;
    g.threads = NT;
    g.smem = (k == kRowFwd || k == kRowInv) ? SM_ROWS : SM_STRIDED;
    return g;
  }
  static cudaError_t r2c(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * W - 1) / (2 * W) * jobs.count;
    auto f = k_r2c_ax0<V, P, W, T>;
    f<<<persistent_grid((const void*)f, NT, SM_STRIDED, tiles), NT, SM_STRIDED, s>>>(jobs, C);
    return cudaGetLastError();
  }
  static cudaError_t rowf(const Jobs& jobs, long long rows, cudaStream_t s) {
    const long long tiles = (rows + W - 1) / W * jobs.count;
    auto f = k_row_fwd<V, P, W, T>;
    f<<<persistent_grid((const void*)f, NT, SM_ROWS, tiles), NT, SM_ROWS, s>>>(jobs, rows);
    return cudaGetLastError();
  }
  static cudaError_t colm(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    const long long tiles = (long long)((M2 + W - 1) / W) * planes * jobs.count;
    auto f = k_col_mid<V, P, W, T>;
    f<<<persistent_grid((const void*)f, NT, SM_STRIDED, tiles), NT, SM_STRIDED, s>>>(jobs, M2, planes);
    return cudaGetLastError();
  }
  static cudaError_t rowi(const Jobs& jobs, long long rows, cudaStream_t s) {
    const long long tiles = (rows + W - 1) / W * jobs.count;
    auto f = k_row_inv<V, P, W, T>;
    f<<<persistent_grid((const void*)f, NT, SM_ROWS, tiles), NT, SM_ROWS, s>>>(jobs, rows);
    return cudaGetLastError();
  }
  static cudaError_t c2r(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * W - 1) / (2 * W) * jobs.count;
    auto f = k_c2r_ax0<V, P, W, T>;
    f<<<persistent_grid((const void*)f, NT, SM_STRIDED, tiles), NT, SM_STRIDED, s>>>(jobs, C);
    return cudaGetLastError();
  }
};

// Second-generation (two-step register) kernels, FP32.
template <int M> struct Inst2 {
  using P = typename Plan2For<M>::type;
  using G = Geo2<P>;
  static constexpr int W = G::W;
  static cudaError_t prepare() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f, int bytes) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    set((const void*)k2_r2c_ax0<P>, G::SM_STRIDED);
    set((const void*)k2_row_fwd<P>, G::SM_ROWS);
    set((const void*)k2_col_mid<P>, G::SM_STRIDED);
    set((const void*)k2_row_inv<P>, G::SM_ROWS);
    set((const void*)k2_c2r_ax0<P>, G::SM_STRIDED);
    return e;
  }
  static Geometry geometry(PassKind k) {
    Geometry g;
    g.W = W;
    g.threads = G::NT;
    g.smem = (k == kRowFwd || k == kRowInv) ? G::SM_ROWS : G::SM_STRIDED;
    return g;
  }
  static cudaError_t r2c(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * W - 1) / (2 * W) * jobs.count;
    auto f = k2_r2c_ax0<P>;
    f<<<persistent_grid((const void*)f, G::NT, G::SM_STRIDED, tiles), G::NT, G::SM_STRIDED, s>>>(jobs, C);
    return cudaGetLastError();
  }
  static cudaError_t rowf(const Jobs& jobs, long long rows, cudaStream_t s) {
    const long long tiles = (rows + W - 1) / W * jobs.count;
    auto f = k2_row_fwd<P>;
    f<<<persistent_grid((const void*)f, G::NT, G::SM_ROWS, tiles), G::NT, G::SM_ROWS, s>>>(jobs, rows);
    return cudaGetLastError();
  }
  static cudaError_t colm(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    const long long tiles = (long long)((M2 + W - 1) / W) * planes * jobs.count;
    auto f = k2_col_mid<P>;
    f<<<persistent_grid((const void*)f, G::NT, G::SM_STRIDED, tiles), G::NT, G::SM_STRIDED, s>>>(jobs, M2,
                                                                                                  planes);
    return cudaGetLastError();
  }
  static cudaError_t rowi(const Jobs& jobs, long long rows, cudaStream_t s) {
    const long long tiles = (rows + W - 1) / W * jobs.count;
    auto f = k2_row_inv<P>;
    f<<<persistent_grid((const void*)f, G::NT, G::SM_ROWS, tiles), G::NT, G::SM_ROWS, s>>>(jobs, rows);
    return cudaGetLastError();
  }
  static cudaError_t c2r(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * W - 1) / (2 * W) * jobs.count;
    auto f = k2_c2r_ax0<P>;
    f<<<persistent_grid((const void*)f, G::NT, G::SM_STRIDED, tiles), G::NT, G::SM_STRIDED, s>>>(jobs, C);
    return cudaGetLastError();
  }
};


}  // namespace detail

#define FSA_DISPATCH(M, CALL)                         \
  switch (M) {                                        \
    case 8: return detail::Inst<V, 8>::CALL;          \
    case 12: return detail::Inst<V, 12>::CALL;        \
    case 16: return detail::Inst<V, 16>::CALL;        \
    case 24: return detail::Inst<V, 24>::CALL;        \
    case 32: return detail::Inst<V, 32>::CALL;        \
    case 48: return detail::Inst<V, 48>::CALL;        \
    case 64: return detail::Inst<V, 64>::CALL;        \
    case 96: return detail::Inst<V, 96>::CALL;        \
    case 128: return detail::Inst<V, 128>::CALL;      \
    case 192: return detail::Inst<V, 192>::CALL;      \
    case 256: return detail::Inst<V, 256>::CALL;      \
    case 384: return detail::Inst<V, 384>::CALL;      \
    case 512: return detail::Inst<V, 512>::CALL;      \
    case 768: return detail::Inst<V, 768>::CALL;      \
    case 1024: return detail::Inst<V, 1024>::CALL;    \
    default: break;                                   \
  }

#define FSA_DISPATCH2(M, CALL)                        \
  switch (M) {                                        \
    case 8: return detail::Inst2<8>::CALL;            \
    case 12: return detail::Inst2<12>::CALL;          \
    case 16: return detail::Inst2<16>::CALL;          \
    case 24: return detail::Inst2<24>::CALL;          \
    case 32: return detail::Inst2<32>::CALL;          \
    case 48: return detail::Inst2<48>::CALL;          \
    case 64: return detail::Inst2<64>::CALL;          \
    case 96: return detail::Inst2<96>::CALL;          \
    case 128: return detail::Inst2<128>::CALL;        \
    case 192: return detail::Inst2<192>::CALL;        \
    case 256: return detail::Inst2<256>::CALL;        \
    case 384: return detail::Inst2<384>::CALL;        \
    case 512: return detail::Inst2<512>::CALL;        \
    case 768: return detail::Inst2<768>::CALL;        \
    case 1024: return detail::Inst2<1024>::CALL;      \
    default: break;                                   \
  }

// FP32 has two kernel generations; the variant table (plan.cu) picks one per
// pass and length.  FP64 has the first generation only.
#define FSA_PICK(KIND, M, CALL)                                         \
  if constexpr (std::is_same<V, float2>::value) {                       \
    if (kernel_variant(KIND, M, FSA_F32) == 2) { FSA_DISPATCH2(M, CALL); } \
  }                                                                     \
  FSA_DISPATCH(M, CALL);

template <typename V> cudaError_t Passes<V>::prepare(int M) {
  if constexpr (std::is_same<V, float2>::value) {
    cudaError_t e = [&]() -> cudaError_t {
      FSA_DISPATCH2(M, prepare());
      return cudaErrorInvalidValue;
    }();
    if (e != cudaSuccess) return e;
  }
  FSA_DISPATCH(M, prepare());
  return cudaErrorInvalidValue;
}
template <typename V> Geometry Passes<V>::geometry(PassKind k, int M) {
  FSA_PICK(k, M, geometry(k));
  return Geometry{};
}
template <typename V>
cudaError_t Passes<V>::r2c_ax0(int M, const Jobs& jobs, long long C, cudaStream_t s) {
  FSA_PICK(kR2C, M, r2c(jobs, C, s));
  return cudaErrorInvalidValue;
}
template <typename V>
cudaError_t Passes<V>::row_fwd(int M, const Jobs& jobs, long long rows, cudaStream_t s) {
  FSA_PICK(kRowFwd, M, rowf(jobs, rows, s));
  return cudaErrorInvalidValue;
}
template <typename V>
cudaError_t Passes<V>::col_mid(int M, const Jobs& jobs, int M2, int planes, cudaStream_t s) {
  FSA_PICK(kColMid, M, colm(jobs, M2, planes, s));
  return cudaErrorInvalidValue;
}
template <typename V>
cudaError_t Passes<V>::row_inv(int M, const Jobs& jobs, long long rows, cudaStream_t s) {
  FSA_PICK(kRowInv, M, rowi(jobs, rows, s));
  return cudaErrorInvalidValue;
}
template <typename V>
cudaError_t Passes<V>::c2r_ax0(int M, const Jobs& jobs, long long C, cudaStream_t s) {
  FSA_PICK(kC2R, M, c2r(jobs, C, s));
  return cudaErrorInvalidValue;
}

template <typename V> cudaError_t Passes<V>::init_twiddles() {
  std::vector<double> re(kTwN), im(kTwN);
  host_twiddles(re.data(), im.data());
  std::vector<float2> t32(kTwN);
  std::vector<double2> t64(kTwN);
  for (int k = 0; k < kTwN; ++k) {
    t32[k] = make_float2((float)re[k], (float)im[k]);
    t64[k] = make_double2(re[k], im[k]);
  }
  cudaError_t e = cudaMemcpyToSymbol(g_tw32, t32.data(), sizeof(float2) * kTwN);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tw64, t64.data(), sizeof(double2) * kTwN);
  return e;
}

#undef FSA_PICK
#undef FSA_DISPATCH2
#undef FSA_DISPATCH

}  // namespace fsa
