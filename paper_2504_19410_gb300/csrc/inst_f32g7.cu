// FP32 seventh-generation passes (passes7.cuh): the row-forward, middle and
// row-inverse passes of a solve as one persistent kernel fed by a work
// dispenser, transform lengths 128 to 512 with n1 = n2.
#include "passes7.cuh"
#include "passes_impl.cuh"

namespace fsa {
namespace {

constexpr int kLagRounds = 4;

template <int M> struct Inst7 {
  using P = typename Plan2For<M>::type;
  using G = Geo7<P>;
  static cudaError_t prepare() {
    return cudaFuncSetAttribute((const void*)k7_pipe<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
  }
  // jobs: in = X, out = Y, S = spectrum octant; job 0's aux = the counters
  // (pipe_ctr_bytes), zeroed here before the launch
  static cudaError_t run(const Jobs& jobs, int n1, int K0, cudaStream_t s) {
    const int a = (n1 + G::W - 1) / G::W, b = M / G::W, c = a;
    const int NP = K0 * jobs.count;
    if (n1 != M / 2 || NP < 2 || !jobs.j[0].aux || (long long)NP * (a + b + c) >= (1LL << 30))
      return cudaErrorInvalidValue;
    auto f = k7_pipe<P>;
    const long long big = 1LL << 40;
    const int resident = persistent_grid((const void*)f, G::NT, G::SMEM, big);
    // lag: every resident CTA holds up to three items (the current one, the
    // next, whose inputs it may be staging, and the one after); a lag of
    // kLagRounds such rounds of the dispenser keeps a plane's row-forward
    // tiles finished before its middle tiles are handed out, and those before
    // its row-inverse tiles
    int L = (kLagRounds * resident + a + b + c - 1) / (a + b + c);
    L = std::max(1, std::min(L, NP / 2));
    const PipeSched sc = make_pipe_sched(a, b, c, NP, L);
    Jobs jj = jobs;
    jj.fault = device_fault_word();
    cudaError_t e = cudaMemsetAsync(const_cast<void*>(jobs.j[0].aux), 0, sizeof(unsigned) * (2 + 2 * (size_t)NP), s);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<long long>(resident, sc.total);
    f<<<grid, G::NT, G::SMEM, s>>>(jj, n1, K0, sc);
    return cudaGetLastError();
  }
};

}  // namespace

PipeFn k7_pipe_fn(int M) {
  switch (M) {
    case 128: return &Inst7<128>::run;
    case 192: return &Inst7<192>::run;
    case 256: return &Inst7<256>::run;
    case 384: return &Inst7<384>::run;
    case 512: return &Inst7<512>::run;
    default: return nullptr;
  }
}

cudaError_t k7_prepare(int M) {
  switch (M) {
    case 128: return Inst7<128>::prepare();
    case 192: return Inst7<192>::prepare();
    case 256: return Inst7<256>::prepare();
    case 384: return Inst7<384>::prepare();
    case 512: return Inst7<512>::prepare();
    default: return cudaSuccess;
  }
}

}  // namespace fsa

// This unit's copy of the twiddle tables (fft_core.cuh) is filled at plan
// creation like every instance unit's: registered here, no pass tables.
FSA_REGISTER()
