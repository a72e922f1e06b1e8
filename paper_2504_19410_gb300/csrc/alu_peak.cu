// fsa_measure_alu_peak: the device's measured FP32 and FP64 fused multiply-add
// rates, the denominators of the ALU rooflines.
//
// The double-word FP64 tier runs on the FP32 pipes and the native FP64 passes
// on the FP64 pipe, so their rooflines are operation rates, not bytes.  This
// measures those rates instead of deriving them from unit counts: every thread
// runs kChains independent fused multiply-add chains (enough to hide the FMA
// latency with the resident warps) for `iters` rounds, and the launch is
// timed with CUDA events.  One FMA is one lane operation (two flops).  The
// kernels touch no memory but one conditional store that keeps the chains
// alive; they have no waits and end after a fixed count of operations.
#include <type_traits>

#include "fsa_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;

// Where a chain's sum would be stored if it ever matched the sentinel (it
// cannot: the chains stay positive); the store keeps the work from being
// removed.
__device__ double g_sink[kThreads];

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T a, T b, int iters) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += x[c];
  if (acc == (T)-1.2345e-7) g_sink[threadIdx.x] = (double)acc;
}

// The same with the paired FP32 instruction of sm_100 and later
// (fma.rn.f32x2: two FP32 FMAs on a register pair, one instruction): each
// chain is a pair, so a thread runs 2 kChains FP32 FMA chains.
__global__ void __launch_bounds__(kThreads) k_fma2_chains(float a, float b, int iters) {
  unsigned long long x[kChains], av, bv;
  asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    const float x0 = (float)(threadIdx.x + c) * 1e-3f, x1 = x0 + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(x0), "f"(x1));
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    }
  }
  float acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    float p, q;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(p), "=f"(q) : "l"(x[c]));
    acc += p + q;
  }
  if (acc == -1.2345e-7f) g_sink[threadIdx.x] = (double)acc;
}

template <typename T>
void launch_chains(int blocks, cudaStream_t s, T a, T b, int iters) {
  k_fma_chains<T><<<blocks, kThreads, 0, s>>>(a, b, iters);
}

struct Pair {};  // selects k_fma2_chains

template <>
void launch_chains<Pair>(int blocks, cudaStream_t s, Pair, Pair, int iters) {
  k_fma2_chains<<<blocks, kThreads, 0, s>>>(0.999999f, 1e-6f, iters);
}

template <typename T>
cudaError_t time_chains(int iters, int blocks, cudaStream_t s, float* best_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // a = slightly below 1, b small: the chains stay finite and normal
  T a{}, b{};
  if constexpr (!std::is_same<T, Pair>::value) {
    a = (T)0.999999;
    b = (T)1e-6;
  }
  *best_ms = 1e30f;
  for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {  // rep 0 warms up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      launch_chains<T>(blocks, s, a, b, iters);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < *best_ms) *best_ms = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" fsa_status fsa_measure_alu_peak(int device, int kind, double* lane_ops_per_s, float* ms) {
  if (!lane_ops_per_s || kind < 0 || kind > 2)
    return fsa::set_error(FSA_ERR_INVALID_ARG,
                          "fsa_measure_alu_peak: kind must be 0 (FP32), 1 (FP64) or 2 (paired FP32)");
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && device >= 0 && device != prev) e = cudaSetDevice(device);
  int dev = 0, sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = kind == 0   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<float>, kThreads, 0)
        : kind == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<double>, kThreads, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma2_chains, kThreads, 0);
  cudaStream_t s = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  // a few ms per launch at the expected rates (FP32 ~40 Tops, FP64 ~1 Tops)
  const int iters = kind == 1 ? 512 : 16384;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  float best = 0;
  if (e == cudaSuccess)
    e = kind == 0   ? time_chains<float>(iters, blocks, s, &best)
        : kind == 1 ? time_chains<double>(iters, blocks, s, &best)
                    : time_chains<Pair>(iters, blocks, s, &best);
  if (s) cudaStreamDestroy(s);
  if (prev >= 0 && device >= 0 && device != prev) cudaSetDevice(prev);
  if (e != cudaSuccess) return fsa::cuda_error(e, "fsa_measure_alu_peak");
  const double ops = (double)blocks * kThreads * iters * 4.0 * kChains * (kind == 2 ? 2 : 1);
  *lane_ops_per_s = ops / (best * 1e-3);
  if (ms) *ms = best;
  return FSA_OK;
}
