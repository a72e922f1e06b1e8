// FP32 sixth-generation middle pass (passes6.cuh), lengths 128 to 512.
// Compiled as its own translation unit; the launchers are looked up by length
// (k6_colm) when the other FP32 instances register their function tables.
#include "passes6.cuh"
#include "passes_impl.cuh"

namespace fsa {
namespace {

template <int M> struct Inst6 {
  using P = typename Plan6For<M>::type;
  static cudaError_t prepare() {
    return cudaFuncSetAttribute((const void*)k6_col_mid<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, P::SMEM);
  }
  static cudaError_t colm(const Jobs& jobs, int M2, int planes, cudaStream_t s) {
    const long long tiles = (long long)((M2 + P::W - 1) / P::W) * planes * jobs.count;
    auto f = k6_col_mid<P>;
    f<<<persistent_grid((const void*)f, P::NT, P::SMEM, tiles), P::NT, P::SMEM, s>>>(jobs, M2, planes);
    return cudaGetLastError();
  }
};

}  // namespace

ColmFn k6_colm(int M) {
  switch (M) {
    case 128: return &Inst6<128>::colm;
    case 192: return &Inst6<192>::colm;
    case 256: return &Inst6<256>::colm;
    case 384: return &Inst6<384>::colm;
    case 512: return &Inst6<512>::colm;
    default: return nullptr;
  }
}

cudaError_t k6_prepare(int M) {
  switch (M) {
    case 128: return Inst6<128>::prepare();
    case 192: return Inst6<192>::prepare();
    case 256: return Inst6<256>::prepare();
    case 384: return Inst6<384>::prepare();
    case 512: return Inst6<512>::prepare();
    default: return cudaSuccess;
  }
}

}  // namespace fsa

// This unit's copy of the twiddle tables (fft_core.cuh) is filled at plan
// creation like every instance unit's: registered here, no pass tables.
FSA_REGISTER()
