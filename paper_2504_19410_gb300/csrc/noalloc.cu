// fsa_apply_noalloc: the apply path with its scratch in a static device array.
//
// fsa_apply keeps its two intermediate arrays (X and Y) in a workspace the
// plan allocated with cudaMalloc.  Some callers cannot have any allocation
// happen on their behalf: a program whose framework's caching allocator has
// already reserved nearly all device memory (a fresh cudaMalloc then fails or
// bypasses its accounting), or a host loop that must not block, since
// cudaMalloc / cudaFree can stall the host and serialise with work already
// running on the device.  This entry point runs the same five passes with X
// and Y placed in g_noalloc_scratch below, a file-scope __device__ array of
// kNoallocScratchBytes that every GPU which loads the library holds until the
// process exits.  It calls no allocating routine.
//
// Set-up: the array's device address is looked up with cudaGetSymbolAddress
// (in host code the array's name is only a host-side stand-in, not a device
// address), once per device, with that device current, and kept.  The lookup
// is also what makes the driver load this file's module and so reserve the
// 16 MiB: the library's modules load lazily, and this one has no kernel that
// could load it earlier.  So plan creation does the lookup (noalloc_resolve,
// once per device, when the first plan is made there): by the time a caller
// applies, the array is held and the apply allocates nothing.  Should that
// lookup fail at plan creation, the first fsa_apply_noalloc call retries it
// and reports the error; that first call should then come before any stream
// capture.
//
// Sharing: every call on a device uses the same array, and it keeps the last
// call's contents.  Nothing in it needs to start at zero (each pass writes
// every element it later reads), but calls that overlap on the GPU race on
// it: issue them on one stream, or order them with events.
#include <cstdio>
#include <mutex>

#include "fsa_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = 16u << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};  // device address of the array, per device

// The array's device address on the current device (dev), looked up once.
cudaError_t resolve_locked(int dev, void** out) {
  if (!g_noalloc_addr[dev]) {
    void* addr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = addr;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

using namespace fsa;

namespace fsa {

cudaError_t noalloc_resolve(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  void* addr = nullptr;
  return resolve_locked(dev, &addr);
}

}  // namespace fsa

extern "C" fsa_status fsa_apply_noalloc(const fsa_plan* p, const void* rho, void* phi, fsa_stream_t stream) {
  if (!p || !rho || !phi) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_noalloc: NULL argument");
  if (!p->generated) return set_error(FSA_ERR_NOT_GENERATED, "fsa_apply_noalloc: call fsa_tensor_generate first");
  if ((((uintptr_t)rho) | ((uintptr_t)phi)) & 15u)
    return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_noalloc: rho and phi must be 16-byte aligned");
  if (p->device < 0 || p->device >= kMaxDevices)
    return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_noalloc: device ordinal out of range");
  const size_t s = p->dtype == FSA_F32 ? 4 : 8;
  const size_t K0 = (size_t)p->n[0] + 1;
  const size_t x_bytes = K0 * p->n[1] * p->n[2] * 2 * s;
  const size_t need = plan_workspace_bytes(p->n, p->dtype);  // X, Y and the pipelined kernel's counters
  if (need > kNoallocScratchBytes) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "fsa_apply_noalloc: grid %dx%dx%d needs %zu scratch bytes; the static scratch holds %zu "
             "(use fsa_apply for this size)",
             p->n[0], p->n[1], p->n[2], need, kNoallocScratchBytes);
    return set_error(FSA_ERR_INVALID_ARG, buf);
  }
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != p->device) e = cudaSetDevice(p->device);
  if (e != cudaSuccess) return cuda_error(e, "fsa_apply_noalloc: cudaSetDevice");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    e = resolve_locked(p->device, &base);
  }
  if (e == cudaSuccess) {
    const void* r[1] = {rho};
    void* f[1] = {phi};
    void* X[1] = {base};
    void* Y[1] = {static_cast<char*>(base) + x_bytes};
    const void* S[1] = {plan_apply_spectrum(p)};
    const DdiPar* par[1] = {p->ddi_par};
    e = run_group(p, 1, r, f, X, Y, S, (cudaStream_t)stream, nullptr, par);
  }
  if (prev != p->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_error(e, "fsa_apply_noalloc");
  return FSA_OK;
}
