// FP32 fused outer pass pairs (passes5.cuh), transform lengths 64, 128, 256,
// 384 and 512 on axes 0 and 2, in their cluster configurations; registers the
// launchers at library load under kArithF32G5.
#include <map>
#include <mutex>

#include "passes5.cuh"
#include "passes_impl.cuh"

namespace fsa {
namespace detail {

// Clusters of one kernel that fit on the device at once (the persistent grid),
// cached per (device, kernel).
int resident_clusters(const void* key, cudaError_t (*query)(int*, int), int smem) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find({dev, key});
  if (it != cache.end()) return it->second;
  int n = 0;
  if (query(&n, smem) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cache[{dev, key}] = n;
  return n;
}

template <int M, int CS, int NT> struct Inst5 {
  static_assert(CS <= 8, "portable cluster sizes only");
  using P = typename Plan2For<M>::type;
  using G = FusedGeo<P, P, CS, NT>;
  static constexpr int kClusterCtas = CS, kThreads = NT;
  static constexpr auto kFwd = k5_fwd<P, P, CS, NT>;
  static constexpr auto kInv = k5_inv<P, P, CS, NT>;

  // shared-memory opt-in, then the resident cluster counts (queried here, at
  // plan creation, not during a stream capture)
  static cudaError_t prepare() {
    cudaError_t e = cudaFuncSetAttribute((const void*)kFwd, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_F);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)kInv, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM_I);
    if (e == cudaSuccess) {
      resident_clusters((const void*)kFwd, &query_fwd, G::SMEM_F);
      resident_clusters((const void*)kInv, &query_inv, G::SMEM_I);
    }
    return e;
  }
  static cudaLaunchConfig_t config(dim3 grid, int smem, cudaStream_t s, cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
  }
  static cudaError_t query_fwd(int* n, int smem) {
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = config(dim3(CS, 1, 1), smem, 0, at);
    return cudaOccupancyMaxActiveClusters(n, kFwd, &cfg);
  }
  static cudaError_t query_inv(int* n, int smem) {
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = config(dim3(CS, 1, 1), smem, 0, at);
    return cudaOccupancyMaxActiveClusters(n, kInv, &cfg);
  }
  // one cluster per slab up to the resident count (persistent beyond it)
  static dim3 grid(const void* key, cudaError_t (*query)(int*, int), int smem, const Jobs& jobs, int n1) {
    const long long slabs = (long long)n1 * jobs.count;
    const int rc = resident_clusters(key, query, smem);
    const long long g = rc < slabs ? rc : slabs;
    return dim3((unsigned)(g * CS), 1, 1);
  }
  static cudaError_t fwd(const Jobs& jobs, int n1, cudaStream_t s) {
    const dim3 g = grid((const void*)kFwd, &query_fwd, G::SMEM_F, jobs, n1);
    if (g.x == 0) return cudaErrorInvalidConfiguration;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = config(g, G::SMEM_F, s, at);
    return cudaLaunchKernelEx(&cfg, kFwd, jobs, n1);
  }
  static cudaError_t inv(const Jobs& jobs, int n1, cudaStream_t s) {
    const dim3 g = grid((const void*)kInv, &query_inv, G::SMEM_I, jobs, n1);
    if (g.x == 0) return cudaErrorInvalidConfiguration;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = config(g, G::SMEM_I, s, at);
    return cudaLaunchKernelEx(&cfg, kInv, jobs, n1);
  }
};

// The configurations of one length, in the order fsa_fused_configs lists them.
template <int M, class... I> struct Fused {
  static cudaError_t prepare() {
    cudaError_t e = cudaSuccess;
    ((e = e == cudaSuccess ? I::prepare() : e), ...);
    return e;
  }
  static cudaError_t fwd(int cfg, const Jobs& jobs, int n1, cudaStream_t s) {
    int k = 0;
    cudaError_t e = cudaErrorInvalidValue;
    ((e = (k++ == cfg) ? I::fwd(jobs, n1, s) : e), ...);
    return e;
  }
  static cudaError_t inv(int cfg, const Jobs& jobs, int n1, cudaStream_t s) {
    int k = 0;
    cudaError_t e = cudaErrorInvalidValue;
    ((e = (k++ == cfg) ? I::inv(jobs, n1, s) : e), ...);
    return e;
  }
  static void add() {
    PassFns f;
    f.prepare = &prepare;
    f.fwd5 = &fwd;
    f.inv5 = &inv;
    int k = 0;
    ((f.fused_cs[k] = I::kClusterCtas, f.fused_nt[k] = I::kThreads, ++k), ...);
    f.nfused = k;
    register_pass_fns(kArithF32G5, M, f);
  }
};

}  // namespace detail
}  // namespace fsa

FSA_REGISTER(
    fsa::detail::Fused<512, fsa::detail::Inst5<512, 8, 128>>::add();
    fsa::detail::Fused<384, fsa::detail::Inst5<384, 4, 128>>::add();
    fsa::detail::Fused<256, fsa::detail::Inst5<256, 4, 256>, fsa::detail::Inst5<256, 8, 128>>::add();
    fsa::detail::Fused<128, fsa::detail::Inst5<128, 4, 64>, fsa::detail::Inst5<128, 2, 64>>::add();
    fsa::detail::Fused<64, fsa::detail::Inst5<64, 2, 64>>::add();
)
