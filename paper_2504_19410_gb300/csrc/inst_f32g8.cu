// FP32 eighth-generation middle, R2C and C2R passes (passes8.cuh): the column
// tiles staged by tiled bulk tensor copies, lengths 128 to 512.  Compiled as
// its own translation unit; the launchers are looked up by length (k8_colm,
// k8_colm_shared, k8_r2c, k8_c2r) when the other FP32 instances register
// their function tables.  A launch whose buffers a tensor map cannot describe
// runs generation 2's kernel for that pass (its registered launcher).
#include <cudaTypedefs.h>

#include <mutex>

#include "passes8.cuh"
#include "passes_impl.cuh"

namespace fsa {
namespace {

// cuTensorMapEncodeTiled from the driver (no link against libcuda).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// A tensor map of one 2-D array: dims {inner, rows} of `esize`-byte elements
// (rows `inner` elements apart), box {box_inner, box_rows}; false if the
// driver cannot encode it (then the caller takes generation 2's kernel).
bool encode_2d(CUtensorMap* map, const void* base, CUtensorMapDataType dt, int esize, long long inner,
               long long rows, int box_inner, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc || reinterpret_cast<uintptr_t>(base) % 16 != 0 || (inner * esize) % 16 != 0 || rows >= (1LL << 31) ||
      inner >= (1LL << 31))
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)inner * esize};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int M> struct Inst8 {
  using P = typename Plan2For<M>::type;
  using G = Geo8<P>;
  using GR = Geo8R<P>;
  using GC = Geo8C<P>;
  static cudaError_t prepare() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f, int bytes) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    set((const void*)k8_col_mid<P, 1>, G::SMEM);
    set((const void*)k8_col_mid<P, kMaxJobs>, G::SMEM);
    set((const void*)k8_col_mid<P, kMaxJobs, true>, G::SMEM);
    set((const void*)k8_r2c_ax0<P, 1>, GR::SMEM);
    set((const void*)k8_r2c_ax0<P, kMaxJobs>, GR::SMEM);
    set((const void*)k8_c2r_ax0<P, 1>, GC::SMEM);
    set((const void*)k8_c2r_ax0<P, kMaxJobs>, GC::SMEM);
    return e;
  }
  // The C2R pass: X of each solve as a {C, n0 + 1} tensor of 8-byte elements.
  template <int NJ> static cudaError_t c2r_n(const Jobs& jobs, long long C, cudaStream_t s) {
    TmapSet<NJ> maps;
    for (int j = 0; j < jobs.count; ++j)
      if (!encode_2d(&maps.m[j], jobs.j[j].in, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, C, M / 2 + 1, 2 * GC::W,
                     GC::ROWS / 2))
        return pass_fns(kArithF32G2, M).c2r(jobs, C, s);
    Jobs jj = jobs;
    jj.fault = device_fault_word();
    const long long tiles = (C + 2 * GC::W - 1) / (2 * GC::W) * jobs.count;
    auto f = k8_c2r_ax0<P, NJ>;
    f<<<persistent_grid((const void*)f, GC::NT, GC::SMEM, tiles), GC::NT, GC::SMEM, s>>>(jj, C, maps);
    return cudaGetLastError();
  }
  static cudaError_t c2r(const Jobs& jobs, long long C, cudaStream_t s) {
    return jobs.count == 1 ? c2r_n<1>(jobs, C, s) : c2r_n<kMaxJobs>(jobs, C, s);
  }
  // The R2C pass: rho of each solve as a {C, n0} tensor of floats.  A rho
  // the copy cannot read (not 16-byte aligned, C not a multiple of 4) sends
  // the launch to generation 2's kernel (its registered launcher, prepared
  // with the other instances), which computes the same values.
  template <int NJ> static cudaError_t r2c_n(const Jobs& jobs, long long C, cudaStream_t s) {
    TmapSet<NJ> maps;
    for (int j = 0; j < jobs.count; ++j)
      if (!encode_2d(&maps.m[j], jobs.j[j].in, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, C, M / 2, 2 * GR::W, M / 2))
        return pass_fns(kArithF32G2, M).r2c(jobs, C, s);
    Jobs jj = jobs;
    jj.fault = device_fault_word();
    const long long tiles = (C + 2 * GR::W - 1) / (2 * GR::W) * jobs.count;
    auto f = k8_r2c_ax0<P, NJ>;
    f<<<persistent_grid((const void*)f, GR::NT, GR::SMEM, tiles), GR::NT, GR::SMEM, s>>>(jj, C, maps);
    return cudaGetLastError();
  }
  static cudaError_t r2c(const Jobs& jobs, long long C, cudaStream_t s) {
    return jobs.count == 1 ? r2c_n<1>(jobs, C, s) : r2c_n<kMaxJobs>(jobs, C, s);
  }
  // The middle pass: Y of each solve as a {M2, planes * n1} tensor of
  // 8-byte elements; the same fallback.
  template <int NJ, bool SHARED = false>
  static cudaError_t colm_n(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    constexpr int n1 = M / 2;
    TmapSet<NJ> maps;
    for (int j = 0; j < jobs.count; ++j)
      if (M2 % G::W != 0 || !encode_2d(&maps.m[j], jobs.j[j].out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, M2,
                                       (long long)planes * n1, G::W, n1))
        return SHARED ? pass_fns(kArithF32G3, M).colm_shared(jobs, M2, planes, s)
                      : pass_fns(kArithF32G2, M).colm(jobs, M2, planes, s);
    Jobs jj = jobs;
    jj.fault = device_fault_word();
    // SHARED: one CTA slot per tile (each walks the tile for every solve)
    const long long tiles = (long long)(M2 / G::W) * planes * (SHARED ? 1 : jobs.count);
    auto f = k8_col_mid<P, NJ, SHARED>;
    f<<<persistent_grid((const void*)f, G::NT, G::SMEM, tiles), G::NT, G::SMEM, s>>>(jj, M2, planes, maps);
    return cudaGetLastError();
  }
  static cudaError_t colm(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    return jobs.count == 1 ? colm_n<1>(jobs, M2, planes, s) : colm_n<kMaxJobs>(jobs, M2, planes, s);
  }
  // densities of one plan: one spectrum read per column tile for all of them
  static cudaError_t colm_shared(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    return colm_n<kMaxJobs, true>(jobs, M2, planes, s);
  }
};

}  // namespace

ColmFn k8_colm_shared(int M) {
  switch (M) {
    case 128: return &Inst8<128>::colm_shared;
    case 192: return &Inst8<192>::colm_shared;
    case 256: return &Inst8<256>::colm_shared;
    case 384: return &Inst8<384>::colm_shared;
    case 512: return &Inst8<512>::colm_shared;
    default: return nullptr;
  }
}

ColmFn k8_colm(int M) {
  switch (M) {
    case 128: return &Inst8<128>::colm;
    case 192: return &Inst8<192>::colm;
    case 256: return &Inst8<256>::colm;
    case 384: return &Inst8<384>::colm;
    case 512: return &Inst8<512>::colm;
    default: return nullptr;
  }
}

R2cFn k8_r2c(int M) {
  switch (M) {
    case 128: return &Inst8<128>::r2c;
    case 192: return &Inst8<192>::r2c;
    case 256: return &Inst8<256>::r2c;
    case 384: return &Inst8<384>::r2c;
    case 512: return &Inst8<512>::r2c;
    default: return nullptr;
  }
}

R2cFn k8_c2r(int M) {
  switch (M) {
    case 128: return &Inst8<128>::c2r;
    case 192: return &Inst8<192>::c2r;
    case 256: return &Inst8<256>::c2r;
    case 384: return &Inst8<384>::c2r;
    case 512: return &Inst8<512>::c2r;
    default: return nullptr;
  }
}

cudaError_t k8_prepare(int M) {
  switch (M) {
    case 128: return Inst8<128>::prepare();
    case 192: return Inst8<192>::prepare();
    case 256: return Inst8<256>::prepare();
    case 384: return Inst8<384>::prepare();
    case 512: return Inst8<512>::prepare();
    default: return cudaSuccess;
  }
}

}  // namespace fsa

// This unit's copy of the twiddle tables (fft_core.cuh) is filled at plan
// creation like every instance unit's: registered here, no pass tables.
FSA_REGISTER()
