// The batched launcher's mixed-length path: every FP32 solve of a batch whose
// transform lengths the mixed kernels carry (passes_mix.cuh) goes through
// five launches in all, one per pass, whatever the mix of grid sizes.
#include <algorithm>
#include <mutex>
#include <set>

#include "fsa_internal.h"
#include "passes_mix.cuh"
#include "passes_impl.cuh"

namespace fsa {
namespace {

std::mutex g_mix_mu;
std::set<int> g_mix_ready;  // devices whose mixed kernels have their shared-memory opt-in

template <int PASS> const void* mix_fn() { return (const void*)k_mix<PASS>; }

cudaError_t mix_prepare() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mix_mu);
  if (g_mix_ready.count(dev)) return cudaSuccess;
  const int smem = mix_smem(512);
  const void* fns[5] = {mix_fn<kMixR2C>(), mix_fn<kMixRowF>(), mix_fn<kMixCol>(), mix_fn<kMixRowI>(),
                        mix_fn<kMixC2R>()};
  for (const void* f : fns)
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) g_mix_ready.insert(dev);
  return e;
}

template <int PASS> cudaError_t launch(const MixJobs& js, int smem, cudaStream_t s) {
  auto f = k_mix<PASS>;
  const long long tiles = js.begin[js.count];
  if (tiles == 0) return cudaSuccess;
  f<<<persistent_grid((const void*)f, kMixNT, smem, tiles), kMixNT, smem, s>>>(js);
  return cudaGetLastError();
}

}  // namespace

bool mixed_eligible(const fsa_plan* p) {
  if (p->dtype != FSA_F32 || p->d != 3 || p->ddi >= 0 || p->chunk_bytes > 0 || !p->ws) return false;
  for (int pass = 0; pass < 5; ++pass)
    if (!mix_supported(mix_length(pass, p->n[0], p->n[1], p->n[2]))) return false;
  return true;
}

cudaError_t mixed_passes(int count, const fsa_plan* const* plans, const void* const* rho, void* const* phi,
                         cudaStream_t s) {
  cudaError_t e = mix_prepare();
  for (int b = 0; b < count && e == cudaSuccess; b += kMaxJobs) {
    const int m = std::min(count - b, kMaxJobs);
    MixJobs js[5];
    int Mmax = 128;
    for (int pass = 0; pass < 5; ++pass) {
      js[pass].count = m;
      js[pass].begin[0] = 0;
    }
    for (int i = 0; i < m; ++i) {
      const fsa_plan* p = plans[b + i];
      void* X = p->ws;
      void* Y = static_cast<char*>(p->ws) + p->x_bytes;
      const void* S = plan_apply_spectrum(p);
      const int n0 = p->n[0], n1 = p->n[1], n2 = p->n[2];
      js[kMixR2C].j[i] = MixJob{rho[b + i], X, nullptr, n0, n1, n2};
      js[kMixRowF].j[i] = MixJob{X, Y, nullptr, n0, n1, n2};
      js[kMixCol].j[i] = MixJob{Y, Y, S, n0, n1, n2};
      js[kMixRowI].j[i] = MixJob{Y, X, nullptr, n0, n1, n2};
      js[kMixC2R].j[i] = MixJob{X, phi[b + i], nullptr, n0, n1, n2};
      for (int pass = 0; pass < 5; ++pass) {
        js[pass].begin[i + 1] = js[pass].begin[i] + mix_tiles(pass, n0, n1, n2);
        Mmax = std::max(Mmax, mix_length(pass, n0, n1, n2));
      }
    }
    const int smem = mix_smem(Mmax);
    if (e == cudaSuccess) e = launch<kMixR2C>(js[kMixR2C], smem, s);
    if (e == cudaSuccess) e = launch<kMixRowF>(js[kMixRowF], smem, s);
    if (e == cudaSuccess) e = launch<kMixCol>(js[kMixCol], smem, s);
    if (e == cudaSuccess) e = launch<kMixRowI>(js[kMixRowI], smem, s);
    if (e == cudaSuccess) e = launch<kMixC2R>(js[kMixC2R], smem, s);
  }
  return e;
}

}  // namespace fsa

// This unit's twiddle tables (fft_core.cuh) are filled at plan creation like
// every instance unit's.
FSA_REGISTER()
