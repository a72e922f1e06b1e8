// Constants shared by host and device code of libfsaconv.
#pragma once

namespace fsa {
// Length of the twiddle table exp(-2 pi i k / kTwN): 3 * 1024 is a multiple
// of every supported transform length 2n (n = 2^a or 3 * 2^a, n <= 512).
constexpr int kTwN = 3072;

// One solve inside a launch: its pass input, pass output and spectrum.
// `par` (3-D DDI plans only): the plan's block of kDdiParCount doubles below;
// `aux`: a second input of the pass (the DDI grid reading's final pass adds
// beta * rho from it).
struct Job {
  const void* in;
  void* out;
  const void* S;
  const void* aux;
  const double* par;
};

// The 3-D DDI multiplier (Sec. 5, Example 4) of one plan, as doubles:
//   D(q) = -(n.mu0)(m.mu0) - (n.nu)(m.nu),  mu_j = w_j q_j,
// q_j the signed DFT frequency of axis j (transform length M_j: q_j in
// [-M_j/2, M_j/2)), mu0 = mu with its Nyquist components (q_j = -M_j/2)
// zeroed, nu = those components alone (nu_j = -w_j M_j/2 = -pi/h_j).  This is
// the real, Hermitian part of the multiplier -(k.n)(k.m), so the real
// inverse transform is exact.  Applied value: cmul * S * D + cadd (kernel
// reading, S the stored spectrum) or cmul * D (grid reading).
enum : int {
  kDdiN = 0,     // n[3]
  kDdiM = 3,     // m[3]
  kDdiW = 6,     // w[3] = 2 pi / (M_j h_j)
  kDdiNu = 9,    // nu[3] = -pi / h_j
  kDdiCmul = 12,
  kDdiCadd = 13,
  kDdiNyq0 = 14,  // axis-0 Nyquist index M_0 / 2 of the pass (the half spectrum's last plane)
  kDdiBeta = 15,  // grid reading: the C2R pass adds beta * rho, beta = -(m.n)
  kDdiParCount = 16
};
constexpr int kMaxJobs = 64;
// The jobs of one launch, passed by value as a kernel parameter (about 2.6 KB):
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
