// Constants shared by host and device code of libfsaconv.
#pragma once

namespace fsa {
// Length of the twiddle table exp(-2 pi i k / kTwN): 3 * 1024 is a multiple
// of every supported transform length 2n (n = 2^a or 3 * 2^a, n <= 512).
constexpr int kTwN = 3072;

// One solve inside a launch: its pass input, pass output and spectrum.
struct Job {
  const void* in;
  void* out;
  const void* S;
};
constexpr int kMaxJobs = 64;
// The jobs of one launch, passed by value as a kernel parameter (about 1.5 KB):
// no device allocation, and a captured CUDA graph keeps its own copy.
// `fault` (device word, may be null): kernels with bounded waits OR a code
// into it when a wait gives up, then return (kWaitTimeout).
struct Jobs {
  Job j[kMaxJobs];
  int count;
  unsigned int* fault;
};
constexpr unsigned int kWaitTimeout = 1u;
// Bound of one wait on an mbarrier, in SM clock cycles (about 1 s).
constexpr long long kWaitLimitCycles = 2000000000LL;
}  // namespace fsa
