// FP32 eighth-generation middle and R2C passes (passes8.cuh): the column
// tiles staged by one tiled bulk tensor copy each, lengths 128 to 512.  Compiled as its own
// translation unit; the launchers are looked up by length (k8_colm) when the
// other FP32 instances register their function tables.
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

template <int M> struct Inst8 {
  using P = typename Plan2For<M>::type;
  using G = Geo8<P>;
  using GR = Geo8R<P>;
  static cudaError_t prepare() {
    cudaError_t e =
        cudaFuncSetAttribute((const void*)k8_col_mid<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)k8_r2c_ax0<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, GR::SMEM);
    return e;
  }
  // The R2C pass of one solve: rho as a {C, n0} tensor of floats (rows of C
  // floats, 16-byte aligned as the copy needs); otherwise generation 2's.
  static cudaError_t r2c(const Jobs& jobs, long long C, cudaStream_t s) {
    constexpr int n0 = M / 2;
    void* rho = const_cast<void*>(jobs.j[0].in);
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (jobs.count != 1 || !enc || C % 4 != 0 || reinterpret_cast<uintptr_t>(rho) % 16 != 0 || C >= (1LL << 31))
      return pass_fns(kArithF32G2, M).r2c(jobs, C, s);
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)C, (cuuint64_t)n0};
    const cuuint64_t strides[1] = {(cuuint64_t)C * 4};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * GR::W), (cuuint32_t)n0};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, rho, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return pass_fns(kArithF32G2, M).r2c(jobs, C, s);
    Jobs jj = jobs;
    jj.fault = device_fault_word();
    const long long tiles = (C + 2 * GR::W - 1) / (2 * GR::W);
    auto f = k8_r2c_ax0<P>;
    f<<<persistent_grid((const void*)f, GR::NT, GR::SMEM, tiles), GR::NT, GR::SMEM, s>>>(jj, C, map);
    return cudaGetLastError();
  }
  // One solve per launch (the tensor map describes its Y); a launch of several
  // solves, or a Y the map cannot describe, runs generation 2's middle pass
  // (its registered launcher, prepared with the other instances), which
  // computes the same values.
  static cudaError_t colm(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    constexpr int n1 = M / 2;
    void* Y = jobs.j[0].out;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (jobs.count != 1 || !enc || M2 % G::W != 0 || reinterpret_cast<uintptr_t>(Y) % 16 != 0 ||
        (long long)planes * n1 >= (1LL << 31))
      return pass_fns(kArithF32G2, M).colm(jobs, M2, planes, s);
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)M2, (cuuint64_t)planes * n1};
    const cuuint64_t strides[1] = {(cuuint64_t)M2 * 8};
    const cuuint32_t box[2] = {(cuuint32_t)G::W, (cuuint32_t)n1};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, Y, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return pass_fns(kArithF32G2, M).colm(jobs, M2, planes, s);
    Jobs jj = jobs;
    jj.fault = device_fault_word();
    const long long tiles = (long long)(M2 / G::W) * planes;
    auto f = k8_col_mid<P>;
    f<<<persistent_grid((const void*)f, G::NT, G::SMEM, tiles), G::NT, G::SMEM, s>>>(jj, M2, planes, map);
    return cudaGetLastError();
  }
};

}  // namespace

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
