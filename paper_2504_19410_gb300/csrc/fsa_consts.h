// Constants shared by host and device code of libfsaconv.
#pragma once

namespace fsa {
// Length of the twiddle table exp(-2 pi i k / kTwN): 3 * 1024 is a multiple
// of every supported transform length 2n (n = 2^a or 3 * 2^a, n <= 512).
constexpr int kTwN = 3072;

struct DdiPar;

// One solve inside a launch: its pass input, pass output and spectrum.
// `par` (3-D DDI plans only): the plan's DDI parameters (DdiPar below);
// `aux`: a second input of the pass (the DDI grid reading's final pass adds
// beta * rho from it).
struct Job {
  const void* in;
  void* out;
  const void* S;
  const void* aux;
  const DdiPar* par;
};

// The 3-D DDI multiplier (Sec. 5, Example 4) of one plan:
//   D(q) = -(n.mu0)(m.mu0) - (n.nu)(m.nu),  mu_j = w_j q_j,
// q_j the signed DFT frequency of axis j (transform length M_j: q_j in
// [-M_j/2, M_j/2)), mu0 = mu with its Nyquist components (q_j = -M_j/2)
// zeroed, nu = those components alone (nu_j = -w_j M_j/2 = -pi/h_j).  This is
// the real, Hermitian part of the multiplier -(k.n)(k.m), so the real
// inverse transform is exact.  Applied value: cmul * S * D + cadd (kernel
// reading, S the stored spectrum) or cmul * D (grid reading).
// Along one middle-pass line (axis 1, fixed axis-0 and axis-2 frequencies)
// cmul D is a quadratic in q1 off its Nyquist index,
//   cmul D = c0 + q1 (c1 + c2 q1),   with a = n.mu0, b = m.mu0 and
//   an = n.nu, bn = m.nu over axes 0 and 2:
//   c0 = -cmul (a b + an bn),  c1 = -cmul (a m1 + b n1) w1,  c2 = -cmul n1 m1 w1^2,
// and at q1 = -M1/2 the constant cN = -cmul (a b + (an + n1 nu1)(bn + m1 nu1)).
// c2 is global (kDdiC2); (c0, c1, cN) per line are tabulated on the host.
enum : int {
  kDdiN = 0,     // n[3]
  kDdiM = 3,     // m[3]
  kDdiW = 6,     // w[3] = 2 pi / (M_j h_j)
  kDdiNu = 9,    // nu[3] = -pi / h_j
  kDdiCmul = 12,
  kDdiCadd = 13,
  kDdiNyq0 = 14,  // axis-0 Nyquist index M_0 / 2 of the pass (the half spectrum's last plane)
  kDdiBeta = 15,  // grid reading: the C2R pass adds beta * rho, beta = -(m.n)
  kDdiC2 = 16,
  kDdiParCount = 17
};

// The parameters in each arithmetic the kernels use, so that no kernel
// converts from FP64 (conversions run on the FP64 pipe, a small fraction of
// the FP32 rate on GB300): d for native FP64, f for FP32, (f, lo) the
// double-word split d = f + lo (to 48 bits).
// `tab`: the per-line coefficients (c0, c1, cN) of the middle pass's lines,
// [k0][k2] for k0 <= nyq0 and k2 < M2, each a triple in the plan's
// arithmetic (float; double; double-word as float pairs).
struct DdiPar {
  double d[kDdiParCount];
  float f[kDdiParCount];
  float lo[kDdiParCount];
  int nyq0;  // = d[kDdiNyq0]
  const void* tab;
};
// The two-step FP32 middle passes walk their tiles from the last (solve,
// plane) to the first.  The row-forward pass before them writes planes in
// ascending order, so the planes it wrote last -- still in the 129 MB L2 --
// are the first ones read (and overwritten in place) here, and the
// row-inverse pass after them, reading in ascending order, starts with the
// planes this pass wrote last (measured at 256^3 with the tensor-copy middle
// pass and the bulk-copy row passes: middle 0.1827 -> 0.1779 ms, row inverse
// 0.0825 -> 0.0799 ms, the solve 0.4067 -> 0.3978 ms).
constexpr bool kMidReverse = true;
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
