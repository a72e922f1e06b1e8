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
template <int PA, int PB> const void* mix2_fn() { return (const void*)k_mix2<PA, PB>; }

cudaError_t mix_prepare() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mix_mu);
  if (g_mix_ready.count(dev)) return cudaSuccess;
  const int smem = mix_smem(512);
  const void* fns[9] = {mix_fn<kMixR2C>(), mix_fn<kMixRowF>(), mix_fn<kMixCol>(), mix_fn<kMixRowI>(),
                        mix_fn<kMixC2R>(), mix2_fn<kMixRowF, kMixR2C>(), mix2_fn<kMixCol, kMixRowF>(),
                        mix2_fn<kMixRowI, kMixCol>(), mix2_fn<kMixC2R, kMixRowI>()};
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

template <int PA, int PB> cudaError_t launch2(const MixJobs& a, const MixJobs& b, int smem, cudaStream_t s) {
  auto f = k_mix2<PA, PB>;
  const long long tiles = a.begin[a.count] + b.begin[b.count];
  if (tiles == 0) return cudaSuccess;
  f<<<persistent_grid((const void*)f, kMixNT, smem, tiles), kMixNT, smem, s>>>(a, b);
  return cudaGetLastError();
}

// The five job tables of `m` solves (plans, rho, phi), and the largest length.
int build_jobs(int m, const fsa_plan* const* plans, const void* const* rho, void* const* phi, MixJobs* js) {
  int Mmax = 128;
  for (int pass = 0; pass < 5; ++pass) {
    js[pass].count = m;
    js[pass].begin[0] = 0;
  }
  for (int i = 0; i < m; ++i) {
    const fsa_plan* p = plans[i];
    void* X = p->ws;
    void* Y = static_cast<char*>(p->ws) + p->x_bytes;
    const void* S = plan_apply_spectrum(p);
    const int n0 = p->n[0], n1 = p->n[1], n2 = p->n[2];
    js[kMixR2C].j[i] = MixJob{rho[i], X, nullptr, n0, n1, n2};
    js[kMixRowF].j[i] = MixJob{X, Y, nullptr, n0, n1, n2};
    js[kMixCol].j[i] = MixJob{Y, Y, S, n0, n1, n2};
    js[kMixRowI].j[i] = MixJob{Y, X, nullptr, n0, n1, n2};
    js[kMixC2R].j[i] = MixJob{X, phi[i], nullptr, n0, n1, n2};
    for (int pass = 0; pass < 5; ++pass) {
      js[pass].begin[i + 1] = js[pass].begin[i] + mix_tiles(pass, n0, n1, n2);
      Mmax = std::max(Mmax, mix_length(pass, n0, n1, n2));
    }
  }
  return Mmax;
}

}  // namespace

bool mixed_eligible(const fsa_plan* p) {
  if (p->dtype != FSA_F32 || p->d != 3 || p->ddi >= 0 || p->chunk_bytes > 0 || !p->ws) return false;
  for (int pass = 0; pass < 5; ++pass)
    if (!mix_supported(mix_length(pass, p->n[0], p->n[1], p->n[2]))) return false;
  return true;
}

int& batched_mode() {
  static int mode = 0;
  return mode;
}

cudaError_t mixed_passes(int count, const fsa_plan* const* plans, const void* const* rho, void* const* phi,
                         cudaStream_t s, bool pipelined) {
  cudaError_t e = mix_prepare();
  for (int b = 0; b < count && e == cudaSuccess; b += 2 * kMaxJobs) {
    const int m = std::min(count - b, 2 * kMaxJobs);
    if (!pipelined || m == 1) {
      // one launch per pass over all the solves' tiles (64 solves per table)
      for (int c = 0; c < m && e == cudaSuccess; c += kMaxJobs) {
        const int mm = std::min(m - c, kMaxJobs);
        MixJobs js[5];
        const int smem = mix_smem(build_jobs(mm, plans + b + c, rho + b + c, phi + b + c, js));
        if (e == cudaSuccess) e = launch<kMixR2C>(js[kMixR2C], smem, s);
        if (e == cudaSuccess) e = launch<kMixRowF>(js[kMixRowF], smem, s);
        if (e == cudaSuccess) e = launch<kMixCol>(js[kMixCol], smem, s);
        if (e == cudaSuccess) e = launch<kMixRowI>(js[kMixRowI], smem, s);
        if (e == cudaSuccess) e = launch<kMixC2R>(js[kMixC2R], smem, s);
      }
      continue;
    }
    // software pipeline over two halves A and B of balanced work: six launches,
    // the middle four each carrying A's pass p and B's pass p - 1
    std::vector<int> order(m);
    for (int i = 0; i < m; ++i) order[i] = i;
    auto work = [&](int i) {
      const fsa_plan* p = plans[b + i];
      return (double)p->n[0] * p->n[1] * p->n[2];
    };
    std::sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
    std::vector<const fsa_plan*> pa, pb;
    std::vector<const void*> ra, rb;
    std::vector<void*> fa, fb;
    double wa = 0, wb = 0;
    for (int i : order) {
      const bool to_a = (wa <= wb && (int)pa.size() < kMaxJobs) || (int)pb.size() >= kMaxJobs;
      (to_a ? pa : pb).push_back(plans[b + i]);
      (to_a ? ra : rb).push_back(rho[b + i]);
      (to_a ? fa : fb).push_back(phi[b + i]);
      (to_a ? wa : wb) += work(i);
    }
    MixJobs A[5], B[5];
    const int smem = mix_smem(std::max(build_jobs((int)pa.size(), pa.data(), ra.data(), fa.data(), A),
                                       build_jobs((int)pb.size(), pb.data(), rb.data(), fb.data(), B)));
    if (e == cudaSuccess) e = launch<kMixR2C>(A[kMixR2C], smem, s);
    if (e == cudaSuccess) e = launch2<kMixRowF, kMixR2C>(A[kMixRowF], B[kMixR2C], smem, s);
    if (e == cudaSuccess) e = launch2<kMixCol, kMixRowF>(A[kMixCol], B[kMixRowF], smem, s);
    if (e == cudaSuccess) e = launch2<kMixRowI, kMixCol>(A[kMixRowI], B[kMixCol], smem, s);
    if (e == cudaSuccess) e = launch2<kMixC2R, kMixRowI>(A[kMixC2R], B[kMixRowI], smem, s);
    if (e == cudaSuccess) e = launch<kMixC2R>(B[kMixC2R], smem, s);
  }
  return e;
}

int mixed_launches(int count, bool pipelined) {
  int n = 0;
  for (int b = 0; b < count; b += 2 * kMaxJobs) {
    const int m = std::min(count - b, 2 * kMaxJobs);
    n += (!pipelined || m == 1) ? 5 * ((m + kMaxJobs - 1) / kMaxJobs) : 6;
  }
  return n;
}

}  // namespace fsa

// This unit's twiddle tables (fft_core.cuh) are filled at plan creation like
// every instance unit's.
FSA_REGISTER()
