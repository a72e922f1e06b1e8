// Host-side launchers of the apply-pass kernel instances, included by the
// instance translation units (inst_*.cu), which register them at load.
#pragma once
#include <mutex>
#include <type_traits>
#include <vector>

#include "fsa_internal.h"
#include "passes.cuh"
#include "passes2.cuh"
#include "passes4.cuh"

namespace fsa {

namespace detail {

template <typename V, int M> struct Inst {
  using P = typename PlanFor<M>::type;
  // the DDI grid reading's unpadded passes (every arithmetic)
  static constexpr bool kUnpadded = true;
  static constexpr int W = TileW<V>::W;
  static constexpr int T = threads_per_line<P, W>();
  static constexpr int NT = W * T;
  static constexpr int SM_STRIDED = smem_strided<P, V, W>();
  static constexpr int SM_ROWS = smem_rows<P, V, W>();
  static constexpr int WC = MidW<V>::W;  // middle pass tile
  static constexpr int TC = threads_per_line<P, WC>();
  static constexpr int NTC = WC * TC;
  static constexpr int SM_MID = smem_strided<P, V, WC>();

  static cudaError_t prepare() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f, int bytes) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    set((const void*)k_r2c_ax0<V, P, W, T>, SM_STRIDED);
    set((const void*)k_row_fwd<V, P, W, T>, SM_ROWS);
    set((const void*)k_col_mid<V, P, WC, TC>, SM_MID);
    set((const void*)k_row_inv<V, P, W, T>, SM_ROWS);
    set((const void*)k_row_mid<V, P, WM, TM>, SM_ROWM);
    set((const void*)k_r2c_ax0<V, P, WM, TM>, SM_STRM);
    set((const void*)k_c2r_ax0<V, P, WM, TM>, SM_STRM);
    set((const void*)k_c2r_ax0<V, P, W, T>, SM_STRIDED);
    set((const void*)k_col_mid<V, P, WC, TC, kMulDdiKernel>, SM_MID);
    set((const void*)k_c2r_ax0<V, P, W, T, true, true>, SM_STRIDED);
    if constexpr (kUnpadded) {
      set((const void*)k_r2c_ax0<V, P, W, T, false>, SM_STRIDED);
      set((const void*)k_row_fwd<V, P, W, T, false>, SM_ROWS);
      set((const void*)k_col_mid<V, P, WC, TC, kMulDdiGrid>, SM_MID);
      set((const void*)k_row_inv<V, P, W, T, false>, SM_ROWS);
      set((const void*)k_c2r_ax0<V, P, W, T, false>, SM_STRIDED);
    }
    return e;
  }
  static Geometry geometry(PassKind k) {
    Geometry g;
    g.W = k == kColMid ? WC : W;
    g.threads = k == kColMid ? NTC : NT;
    g.smem = (k == kRowFwd || k == kRowInv) ? SM_ROWS : (k == kColMid ? SM_MID : SM_STRIDED);
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
    const long long tiles = (long long)((M2 + WC - 1) / WC) * planes * jobs.count;
    auto f = k_col_mid<V, P, WC, TC>;
    f<<<persistent_grid((const void*)f, NTC, SM_MID, tiles), NTC, SM_MID, s>>>(jobs, M2, planes);
    return cudaGetLastError();
  }
  // the d = 2 middle pass: rows of the R2C output, in place.  A plane has
  // only n0 + 1 rows, so its tiles are narrower than the 3-D row passes'
  // (more CTAs for one solve).
  static constexpr int WM = std::is_same<V, float2>::value ? 4 : 2;
  static constexpr int TM = threads_per_line<P, WM>();
  static constexpr int NTM = WM * TM;
  static constexpr int SM_ROWM = smem_rows<P, V, WM>();
  static cudaError_t rowm(const Jobs& jobs, long long rows, cudaStream_t s) {
    const long long tiles = (rows + WM - 1) / WM * jobs.count;
    auto f = k_row_mid<V, P, WM, TM>;
    f<<<persistent_grid((const void*)f, NTM, SM_ROWM, tiles), NTM, SM_ROWM, s>>>(jobs, rows);
    return cudaGetLastError();
  }
  // the plane's R2C / C2R passes: its n1 real columns are few, so narrow tiles
  static constexpr int SM_STRM = smem_strided<P, V, WM>();
  static cudaError_t r2c_plane(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * WM - 1) / (2 * WM) * jobs.count;
    auto f = k_r2c_ax0<V, P, WM, TM>;
    f<<<persistent_grid((const void*)f, NTM, SM_STRM, tiles), NTM, SM_STRM, s>>>(jobs, C);
    return cudaGetLastError();
  }
  static cudaError_t c2r_plane(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * WM - 1) / (2 * WM) * jobs.count;
    auto f = k_c2r_ax0<V, P, WM, TM>;
    f<<<persistent_grid((const void*)f, NTM, SM_STRM, tiles), NTM, SM_STRM, s>>>(jobs, C);
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

  // 3-D DDI (Sec. 5, Example 4).  Kernel reading: the middle pass with the
  // multiplier cmul * S * D + cadd.  Grid reading: the C2R pass adding
  // beta * rho, and the five passes of the unpadded transform of length M
  // (this instance's length is the grid's n there) whose middle multiplies by
  // cmul * D.
  static cudaError_t colm_ddi(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    const long long tiles = (long long)((M2 + WC - 1) / WC) * planes * jobs.count;
    auto f = k_col_mid<V, P, WC, TC, kMulDdiKernel>;
    f<<<persistent_grid((const void*)f, NTC, SM_MID, tiles), NTC, SM_MID, s>>>(jobs, M2, planes);
    return cudaGetLastError();
  }
  static cudaError_t c2r_epi(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * W - 1) / (2 * W) * jobs.count;
    auto f = k_c2r_ax0<V, P, W, T, true, true>;
    f<<<persistent_grid((const void*)f, NT, SM_STRIDED, tiles), NT, SM_STRIDED, s>>>(jobs, C);
    return cudaGetLastError();
  }
  static cudaError_t r2c_per(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * W - 1) / (2 * W) * jobs.count;
    auto f = k_r2c_ax0<V, P, W, T, false>;
    f<<<persistent_grid((const void*)f, NT, SM_STRIDED, tiles), NT, SM_STRIDED, s>>>(jobs, C);
    return cudaGetLastError();
  }
  static cudaError_t rowf_per(const Jobs& jobs, long long rows, cudaStream_t s) {
    const long long tiles = (rows + W - 1) / W * jobs.count;
    auto f = k_row_fwd<V, P, W, T, false>;
    f<<<persistent_grid((const void*)f, NT, SM_ROWS, tiles), NT, SM_ROWS, s>>>(jobs, rows);
    return cudaGetLastError();
  }
  static cudaError_t colm_per(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    const long long tiles = (long long)((M2 + WC - 1) / WC) * planes * jobs.count;
    auto f = k_col_mid<V, P, WC, TC, kMulDdiGrid>;
    f<<<persistent_grid((const void*)f, NTC, SM_MID, tiles), NTC, SM_MID, s>>>(jobs, M2, planes);
    return cudaGetLastError();
  }
  static cudaError_t rowi_per(const Jobs& jobs, long long rows, cudaStream_t s) {
    const long long tiles = (rows + W - 1) / W * jobs.count;
    auto f = k_row_inv<V, P, W, T, false>;
    f<<<persistent_grid((const void*)f, NT, SM_ROWS, tiles), NT, SM_ROWS, s>>>(jobs, rows);
    return cudaGetLastError();
  }
  static cudaError_t c2r_per(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * W - 1) / (2 * W) * jobs.count;
    auto f = k_c2r_ax0<V, P, W, T, false>;
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
    set((const void*)k2p_col_mid<P>, G::SM_STRIDED + Stage2<P>::BYTES);
    set((const void*)k2p_row_fwd<P, 16>, RowGeo<P, 16>::SM_FWD);
    set((const void*)k2p_row_inv<P, 8>, RowGeo<P, 8>::SM_INV);
    set((const void*)k4_row_fwd<P, WRF>, GF::SMEM);
    set((const void*)k4_row_inv<P, WRI>, GI::SMEM);
    set((const void*)k2_col_mid<P, kMulDdiKernel>, G::SM_STRIDED);
    set((const void*)k2p_col_mid<P, kMulDdiKernel>, G::SM_STRIDED + Stage2<P>::BYTES);
    set((const void*)k2p_col_mid<P, kMulSpectrum, true>, G::SM_STRIDED + Stage2<P>::BYTES);
    set((const void*)k2_c2r_ax0<P, true>, G::SM_STRIDED);
    set((const void*)k2_r2c_ax0<P, false>, G::SM_STRIDED);
    set((const void*)k4_row_fwd<P, WRF, false>, GFU::SMEM);
    set((const void*)k2_col_mid<P, kMulDdiGrid>, G::SM_STRIDED);
    set((const void*)k4_row_inv<P, WRI, false>, GI::SMEM);
    set((const void*)k2_c2r_ax0<P, false, false>, G::SM_STRIDED);
    return e;
  }
  // bulk-copy row passes: rows per tile, fewer for the longest lines
  static constexpr int WRF = 4;
  static constexpr int WRI = M >= 1024 ? 4 : 8;
  using GF = BulkGeo<P, WRF, M / 2>;
  using GI = BulkGeo<P, WRI, M>;
  using GFU = BulkGeo<P, WRF, M>;  // unpadded forward rows: M inputs
  static constexpr bool kUnpadded = true;
  // bulk copies need 16-byte aligned sources (row offsets are: n is even)
  static bool inputs_aligned(const Jobs& jobs) {
    for (int i = 0; i < jobs.count; ++i)
      if (reinterpret_cast<uintptr_t>(jobs.j[i].in) % 16 != 0) return false;
    return true;
  }
  static cudaError_t rowf_b(const Jobs& jobs, long long rows, cudaStream_t s) {
    if (!inputs_aligned(jobs)) return rowf_p(jobs, rows, s);
    Jobs jj = jobs;
    jj.fault = device_fault_word();
    const long long tiles = (rows + WRF - 1) / WRF * jobs.count;
    auto f = k4_row_fwd<P, WRF>;
    f<<<persistent_grid((const void*)f, GF::NT, GF::SMEM, tiles), GF::NT, GF::SMEM, s>>>(jj, rows);
    return cudaGetLastError();
  }
  static cudaError_t rowi_b(const Jobs& jobs, long long rows, cudaStream_t s) {
    if (!inputs_aligned(jobs)) return rowi_p(jobs, rows, s);
    Jobs jj = jobs;
    jj.fault = device_fault_word();
    const long long tiles = (rows + WRI - 1) / WRI * jobs.count;
    auto f = k4_row_inv<P, WRI>;
    f<<<persistent_grid((const void*)f, GI::NT, GI::SMEM, tiles), GI::NT, GI::SMEM, s>>>(jj, rows);
    return cudaGetLastError();
  }
  static cudaError_t rowf_p(const Jobs& jobs, long long rows, cudaStream_t s) {
    using RG = RowGeo<P, 16>;
    const long long tiles = (rows + 15) / 16 * jobs.count;
    auto f = k2p_row_fwd<P, 16>;
    f<<<persistent_grid((const void*)f, RG::NT, RG::SM_FWD, tiles), RG::NT, RG::SM_FWD, s>>>(jobs, rows);
    return cudaGetLastError();
  }
  static cudaError_t rowi_p(const Jobs& jobs, long long rows, cudaStream_t s) {
    using RG = RowGeo<P, 8>;
    const long long tiles = (rows + 7) / 8 * jobs.count;
    auto f = k2p_row_inv<P, 8>;
    f<<<persistent_grid((const void*)f, RG::NT, RG::SM_INV, tiles), RG::NT, RG::SM_INV, s>>>(jobs, rows);
    return cudaGetLastError();
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
  static cudaError_t colm_p(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    const long long tiles = (long long)((M2 + W - 1) / W) * planes * jobs.count;
    constexpr int smem = G::SM_STRIDED + Stage2<P>::BYTES;
    auto f = k2p_col_mid<P>;
    f<<<persistent_grid((const void*)f, G::NT, smem, tiles), G::NT, smem, s>>>(jobs, M2, planes);
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
  // 3-D DDI: the kernel reading's middle pass and the grid reading's C2R
  static cudaError_t colm_ddi(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    const long long tiles = (long long)((M2 + W - 1) / W) * planes * jobs.count;
    auto f = k2_col_mid<P, kMulDdiKernel>;
    f<<<persistent_grid((const void*)f, G::NT, G::SM_STRIDED, tiles), G::NT, G::SM_STRIDED, s>>>(jobs, M2,
                                                                                                  planes);
    return cudaGetLastError();
  }
  // densities of one plan: one spectrum read per column tile for all of them
  static cudaError_t colm_p_shared(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    const long long tiles = (long long)((M2 + W - 1) / W) * planes;
    constexpr int smem = G::SM_STRIDED + Stage2<P>::BYTES;
    auto f = k2p_col_mid<P, kMulSpectrum, true>;
    f<<<persistent_grid((const void*)f, G::NT, smem, tiles), G::NT, smem, s>>>(jobs, M2, planes);
    return cudaGetLastError();
  }
  static cudaError_t colm_p_ddi(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    const long long tiles = (long long)((M2 + W - 1) / W) * planes * jobs.count;
    constexpr int smem = G::SM_STRIDED + Stage2<P>::BYTES;
    auto f = k2p_col_mid<P, kMulDdiKernel>;
    f<<<persistent_grid((const void*)f, G::NT, smem, tiles), G::NT, smem, s>>>(jobs, M2, planes);
    return cudaGetLastError();
  }
  static cudaError_t c2r_epi(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * W - 1) / (2 * W) * jobs.count;
    auto f = k2_c2r_ax0<P, true>;
    f<<<persistent_grid((const void*)f, G::NT, G::SM_STRIDED, tiles), G::NT, G::SM_STRIDED, s>>>(jobs, C);
    return cudaGetLastError();
  }
  // the DDI grid reading's unpadded passes of length M (this instance's M is
  // the grid's n there).  Their buffers are the plan's workspace regions,
  // 16-byte aligned by construction, as the bulk row copies need.
  static cudaError_t r2c_per(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * W - 1) / (2 * W) * jobs.count;
    auto f = k2_r2c_ax0<P, false>;
    f<<<persistent_grid((const void*)f, G::NT, G::SM_STRIDED, tiles), G::NT, G::SM_STRIDED, s>>>(jobs, C);
    return cudaGetLastError();
  }
  static cudaError_t rowf_per(const Jobs& jobs, long long rows, cudaStream_t s) {
    if (!inputs_aligned(jobs)) return cudaErrorInvalidValue;
    Jobs jj = jobs;
    jj.fault = device_fault_word();
    const long long tiles = (rows + WRF - 1) / WRF * jobs.count;
    auto f = k4_row_fwd<P, WRF, false>;
    f<<<persistent_grid((const void*)f, GFU::NT, GFU::SMEM, tiles), GFU::NT, GFU::SMEM, s>>>(jj, rows);
    return cudaGetLastError();
  }
  static cudaError_t colm_per(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    const long long tiles = (long long)((M2 + W - 1) / W) * planes * jobs.count;
    auto f = k2_col_mid<P, kMulDdiGrid>;
    f<<<persistent_grid((const void*)f, G::NT, G::SM_STRIDED, tiles), G::NT, G::SM_STRIDED, s>>>(jobs, M2,
                                                                                                  planes);
    return cudaGetLastError();
  }
  static cudaError_t rowi_per(const Jobs& jobs, long long rows, cudaStream_t s) {
    if (!inputs_aligned(jobs)) return cudaErrorInvalidValue;
    Jobs jj = jobs;
    jj.fault = device_fault_word();
    const long long tiles = (rows + WRI - 1) / WRI * jobs.count;
    auto f = k4_row_inv<P, WRI, false>;
    f<<<persistent_grid((const void*)f, GI::NT, GI::SMEM, tiles), GI::NT, GI::SMEM, s>>>(jj, rows);
    return cudaGetLastError();
  }
  static cudaError_t c2r_per(const Jobs& jobs, long long C, cudaStream_t s) {
    const long long tiles = (C + 2 * W - 1) / (2 * W) * jobs.count;
    auto f = k2_c2r_ax0<P, false, false>;
    f<<<persistent_grid((const void*)f, G::NT, G::SM_STRIDED, tiles), G::NT, G::SM_STRIDED, s>>>(jobs, C);
    return cudaGetLastError();
  }
};


}  // namespace detail

// Launchers of one instance as a function table (see fsa_internal.h).
template <class I, class = void> struct HasRowm : std::false_type {};
template <class I> struct HasRowm<I, std::void_t<decltype(&I::rowm)>> : std::true_type {};
template <class I, class = void> struct HasUnpadded : std::false_type {};
template <class I> struct HasUnpadded<I, std::void_t<decltype(I::kUnpadded)>> : std::bool_constant<I::kUnpadded> {};

template <class I> PassFns fns_of() {
  PassFns f;
  if constexpr (HasRowm<I>::value) {
    f.rowm = &I::rowm;
    f.r2c_plane = &I::r2c_plane;
    f.c2r_plane = &I::c2r_plane;
  }
  if constexpr (HasUnpadded<I>::value) {
    f.r2c_per = &I::r2c_per;
    f.rowf_per = &I::rowf_per;
    f.colm_per = &I::colm_per;
    f.rowi_per = &I::rowi_per;
    f.c2r_per = &I::c2r_per;
  }
  f.colm_ddi = &I::colm_ddi;
  f.c2r_epi = &I::c2r_epi;
  f.colm_shared = &I::colm;
  f.prepare = &I::prepare;
  f.geometry = &I::geometry;
  f.r2c = &I::r2c;
  f.rowf = &I::rowf;
  f.colm = &I::colm;
  f.rowi = &I::rowi;
  f.c2r = &I::c2r;
  return f;
}

// Fills this translation unit's copies of the twiddle tables on the current
// device.  Internal linkage on purpose: every unit has its own tables, and an
// external-linkage (inline) definition would be merged into one by the linker.
static cudaError_t init_tu_twiddles() {
  std::vector<double> re(kTwN), im(kTwN);
  host_twiddles(re.data(), im.data());
  std::vector<float2> t32(kTwN);
  std::vector<double2> t64(kTwN);
  std::vector<cdw> tdw(kTwN);
  for (int k = 0; k < kTwN; ++k) {
    t32[k] = make_float2((float)re[k], (float)im[k]);
    t64[k] = make_double2(re[k], im[k]);
    tdw[k] = cdw{dw(re[k]), dw(im[k])};
  }
  cudaError_t e = cudaMemcpyToSymbol(g_tw32, t32.data(), sizeof(float2) * kTwN);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tw64, t64.data(), sizeof(double2) * kTwN);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_twdw, tdw.data(), sizeof(cdw) * kTwN);
  return e;
}

}  // namespace fsa

// Registers the instances of one translation unit at library load.
#define FSA_REGISTER(...)                                                   \
  namespace {                                                              \
  struct Registrar {                                                       \
    Registrar() {                                                          \
      fsa::register_twiddle_init(&fsa::init_tu_twiddles);                  \
      __VA_ARGS__                                                          \
    }                                                                      \
  } registrar_instance;                                                    \
  }
#define FSA_REG_V1(ARITH, V, M) fsa::register_pass_fns(ARITH, M, fsa::fns_of<fsa::detail::Inst<V, M>>());
#define FSA_REG_V2(M)                                                                 \
  {                                                                                   \
    /* densities of one plan: the prefetching middle pass, whichever the     */      \
    /* tuner picks for single solves (it overlaps loads across the densities) */     \
    fsa::PassFns f2 = fsa::fns_of<fsa::detail::Inst2<M>>();                           \
    f2.colm_shared = &fsa::detail::Inst2<M>::colm_p_shared;                           \
    fsa::register_pass_fns(fsa::kArithF32G2, M, f2);                                  \
  }                                                                                   \
  {                                                                                   \
    fsa::PassFns f3 = fsa::fns_of<fsa::detail::Inst2<M>>();                           \
    f3.colm = &fsa::detail::Inst2<M>::colm_p;                                         \
    f3.colm_ddi = &fsa::detail::Inst2<M>::colm_p_ddi;                                 \
    f3.colm_shared = &fsa::detail::Inst2<M>::colm_p_shared;                           \
    f3.rowf = &fsa::detail::Inst2<M>::rowf_p;                                         \
    f3.rowi = &fsa::detail::Inst2<M>::rowi_p;                                         \
    fsa::register_pass_fns(fsa::kArithF32G3, M, f3);                                  \
    f3.rowf = &fsa::detail::Inst2<M>::rowf_b;                                         \
    f3.rowi = &fsa::detail::Inst2<M>::rowi_b;                                         \
    fsa::register_pass_fns(fsa::kArithF32G4, M, f3);                                  \
    /* generation 8: generation 4 with the tensor-copy middle, R2C, C2R passes */     \
    /* where they have an instance (inst_f32g8.cu), generation 4's elsewhere */        \
    {                                                                                 \
      fsa::PassFns f8 = f3;                                                           \
      if (fsa::ColmFn c8 = fsa::k8_colm(M)) f8.colm = c8;                             \
      if (fsa::ColmFn s8 = fsa::k8_colm_shared(M)) f8.colm_shared = s8;               \
      if (fsa::R2cFn r8 = fsa::k8_r2c(M)) f8.r2c = r8;                                \
      if (fsa::R2cFn c8 = fsa::k8_c2r(M)) f8.c2r = c8;                                \
      fsa::register_pass_fns(fsa::kArithF32G8, M, f8);                                \
    }                                                                                 \
    /* generation 6: generation 4 with the low-register middle pass where  */        \
    /* it has an instance (inst_f32g6.cu), generation 4's elsewhere         */        \
    if (fsa::ColmFn c6 = fsa::k6_colm(M)) f3.colm = c6;                               \
    fsa::register_pass_fns(fsa::kArithF32G6, M, f3);                                  \
  }
