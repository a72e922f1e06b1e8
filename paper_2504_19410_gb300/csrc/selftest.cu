// fsa_wait_selftest: exercises the bounded device-side wait.
//
// The generation-4 row passes wait on an mbarrier for their own bulk copies;
// every such wait is bounded, and a CTA that gives up records kWaitTimeout in
// the device's fault word and returns.  Those copies always complete, so the
// path that gives up never runs in a solve.  This entry point runs it on
// purpose: one CTA waits, with a short bound, on an mbarrier that nothing
// arrives on, takes the give-up path of the row passes (record, return), and
// the host reads the word back.  Nothing faults, traps or hangs: the wait
// ends by its bound and the kernel returns normally.
#include "fsa_internal.h"
#include "mbar.cuh"

namespace {

__global__ void k_wait_selftest(unsigned int* fault, long long limit) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    fsa::mbar_init(&bar, 1);  // one arrival expected; none ever comes
    fsa::fence_mbar_init();
  }
  __syncthreads();
  const bool late = !fsa::mbar_wait(&bar, 0, limit);
  if (__syncthreads_or(late) && threadIdx.x == 0 && fault) atomicOr(fault, fsa::kWaitTimeout);
}

}  // namespace

extern "C" fsa_status fsa_wait_selftest(int device, unsigned int* code) {
  if (!code) return fsa::set_error(FSA_ERR_INVALID_ARG, "fsa_wait_selftest: NULL code");
  *code = 0;
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && device >= 0 && device != prev) e = cudaSetDevice(device);
  unsigned int* w = e == cudaSuccess ? fsa::ensure_device_fault_word() : nullptr;
  if (e == cudaSuccess && !w) e = cudaErrorMemoryAllocation;
  cudaStream_t s = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, s>>>(w, 2000000LL);  // about 1 ms of SM clock
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(code, w, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (s) cudaStreamDestroy(s);
  if (prev >= 0 && device >= 0 && device != prev) cudaSetDevice(prev);
  if (e != cudaSuccess) return fsa::cuda_error(e, "fsa_wait_selftest");
  return FSA_OK;
}
