// Plans, validation and the single-solve apply path of libfsaconv.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <tuple>
#include <type_traits>
#include <mutex>
#include <vector>
#include <set>
#include <string>

#include "dw.cuh"
#include "fsa_internal.h"
#include "quad.h"

namespace fsa {

namespace {
thread_local std::string t_last_error;
std::mutex g_init_mu;
std::set<std::pair<int, int>> g_prepared;  // (device, key) pairs already prepared
std::set<int> g_tw_ready;                  // devices with twiddle tables filled
constexpr int kMaxDevices = 64;
unsigned int* g_fault[kMaxDevices] = {};    // per-device fault word (Jobs::fault)
}  // namespace

// Allocates the device's fault word once (device current, g_init_mu held).
cudaError_t ensure_fault_word_locked(int dev) {
  if (dev < 0 || dev >= kMaxDevices || g_fault[dev]) return cudaSuccess;
  unsigned int* w = nullptr;
  cudaError_t e = cudaMalloc(&w, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(w, 0, sizeof(unsigned int));
  if (e != cudaSuccess) return e;
  g_fault[dev] = w;
  return cudaSuccess;
}

unsigned int* ensure_device_fault_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (ensure_fault_word_locked(dev) != cudaSuccess) return nullptr;
  return g_fault[dev];
}

unsigned int* device_fault_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  return g_fault[dev];
}

fsa_status set_error(fsa_status st, const std::string& msg) {
  t_last_error = msg;
  return st;
}

fsa_status cuda_error(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) return set_error(FSA_ERR_OOM, m);
  return set_error(FSA_ERR_CUDA, m);
}

int& launch_grid_mode() {
  static thread_local int mode = 0;
  return mode;
}

int persistent_grid(const void* func, int threads, int smem, long long tiles) {
  if (launch_grid_mode() == 1) return (int)std::max<long long>(1, std::min<long long>(tiles, 1LL << 30));
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> occ;
  static std::map<int, int> sms;
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = 1, nsm = 1;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, func);
    auto it = occ.find(key);
    if (it == occ.end()) {
      int b = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, func, threads, smem) != cudaSuccess || b < 1) b = 1;
      it = occ.emplace(key, b).first;
    }
    per_sm = it->second;
    auto is = sms.find(dev);
    if (is == sms.end()) {
      int c = 0;
      if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c < 1) c = 1;
      is = sms.emplace(dev, c).first;
    }
    nsm = is->second;
  }
  const long long cap = (long long)per_sm * nsm;
  const long long g = tiles < cap ? tiles : cap;
  return (int)(g < 1 ? 1 : g);
}

int& autotune_mode() {
  static int mode = 1;
  return mode;
}

namespace {
// Chosen generation per (pass, transform length, dtype); 0 = not chosen yet.
std::atomic<signed char> g_variant[kNumPass][1025][2];
std::mutex g_tune_mu;
}  // namespace

int kernel_variant(int pass, int M, fsa_dtype dt) {
  const int mode = autotune_mode();
  if (dt == FSA_F64) return 1;
  if (mode == 2) return 1;
  if (mode == 3) return 2;
  if (mode == 4) return 3;
  if (mode == 5) return 4;
  if (mode == 6) return pass == kColMid ? 5 : 4;
  if (mode == 7) return 6;  // generation 8's table: generation 4 elsewhere
  const int v = (M >= 0 && M <= 1024) ? g_variant[pass][M][dt].load(std::memory_order_relaxed) : 0;
  return v ? v : 2;
}

void set_kernel_variant(int pass, int M, fsa_dtype dt, int variant) {
  if (M >= 0 && M <= 1024) g_variant[pass][M][dt].store((signed char)variant, std::memory_order_relaxed);
}

namespace {
// Fused outer pair per (length, direction): -1 unpinned and untuned, else as
// fused_config.  Pins (fsa_fused_select) and tuner results share the table.
std::atomic<signed char> g_fused[1025][2];
std::atomic<bool> g_fused_init{false};
void fused_table_init() {
  if (g_fused_init.load()) return;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (g_fused_init.load()) return;
  for (auto& m : g_fused)
    for (auto& d : m) d.store(-1);
  g_fused_init.store(true);
}
}  // namespace

int fused_config(int M, int dir) {
  const int mode = autotune_mode();
  if (mode >= 2 || M < 0 || M > 1024 || dir < 0 || dir > 1) return 0;
  const int nf = pass_fns(kArithF32G5, M).nfused;
  if (nf == 0) return 0;
  fused_table_init();
  const int c = g_fused[M][dir].load(std::memory_order_relaxed);
  return c >= 0 && c <= nf ? c : 0;  // unpinned and untuned: the separate passes
}

void set_fused_config(int M, int dir, int c) {
  if (M < 0 || M > 1024 || dir < 0 || dir > 1) return;
  fused_table_init();
  g_fused[M][dir].store((signed char)c, std::memory_order_relaxed);
}

namespace {
// Seventh generation per transform length: -1 unpinned, else as pipe_config
// (fsa_pipe_select).
std::atomic<signed char> g_pipe[1025];
std::once_flag g_pipe_once;
void pipe_table_init() {
  std::call_once(g_pipe_once, [] {
    for (auto& c : g_pipe) c.store(-1);
  });
}
}  // namespace

int pipe_config(int M) {
  if (autotune_mode() >= 2 || M < 0 || M > 1024 || !k7_pipe_fn(M)) return 0;
  pipe_table_init();
  return g_pipe[M].load(std::memory_order_relaxed) == 1 ? 1 : 0;
}

void set_pipe_config(int M, int c) {
  if (M < 0 || M > 1024) return;
  pipe_table_init();
  g_pipe[M].store((signed char)(c < -1 ? -1 : c > 1 ? 1 : c), std::memory_order_relaxed);
}

bool supported_n(int n) {
  if (n < 4 || n > 512 || (n & 1)) return false;
  int m = n;
  if (m % 3 == 0) m /= 3;
  return (m & (m - 1)) == 0;  // power of two
}

bool supported_M(int M) { return (M % 2 == 0) && supported_n(M / 2); }

// exp(-2 pi i k / 3072) evaluated in long double and rounded once.
void host_twiddles(double* re, double* im) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < kTwN; ++k) {
    const long double a = 2.0L * pi * (long double)k / (long double)kTwN;
    re[k] = (double)cosl(a);
    im[k] = -(double)sinl(a);
  }
}

}  // namespace fsa

using namespace fsa;

namespace fsa {

// The five passes for `count` solves that share the grid n and the dtype V.
namespace {
PassFns g_fns[kNumArith][1025];
cudaError_t (*g_tw_inits[64])() = {};
int g_ntw = 0;
}  // namespace

void register_pass_fns(int arith, int M, PassFns f) {
  if (arith >= 0 && arith < kNumArith && M >= 0 && M <= 1024) g_fns[arith][M] = f;
}

const PassFns& pass_fns(int arith, int M) {
  static const PassFns none{};
  return (arith >= 0 && arith < kNumArith && M >= 0 && M <= 1024) ? g_fns[arith][M] : none;
}

void register_twiddle_init(cudaError_t (*init)()) {
  if (g_ntw < 64) g_tw_inits[g_ntw++] = init;
}

cudaError_t init_all_twiddles() {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < g_ntw && e == cudaSuccess; ++i) e = g_tw_inits[i]();
  return e;
}

// FP32 kernel variant (1..5, as kernel_variant) -> registered arithmetic.
int arith_of_variant(int v) {
  return v == 6   ? kArithF32G8
         : v == 5 ? kArithF32G6
         : v == 4 ? kArithF32G4
                  : (v == 3 ? kArithF32G3 : (v == 2 ? kArithF32G2 : kArithF32G1));
}

template <typename V> int arith_for(int pass, int M) {
  if constexpr (std::is_same<V, float2>::value) {
    return arith_of_variant(kernel_variant(pass, M, FSA_F32));
  }
  else if constexpr (std::is_same<V, double2>::value)
    return kArithF64;
  else
    return kArithDW;
}

// The three middle passes (row forward, middle, row inverse) of planes
// [k0s, k0s + pc) of every job: the kernels take any count of rows / planes,
// so a slab is the same launch with offset pointers.
cudaError_t trace_mark(PassTrace* tr, int kind, cudaStream_t s) {
  if (!tr || tr->used >= tr->cap) return cudaSuccess;
  if (tr->used > 0) tr->kind[tr->used - 1] = (signed char)kind;
  return cudaEventRecord(tr->ev[tr->used++], s);
}

template <typename V>
cudaError_t middle_slab(const int* n, int m, int b, void* const* X, void* const* Y, const void* const* S, int k0s,
                        int pc, const PassFns& f2, const PassFns& f3, const PassFns& f4, cudaStream_t s,
                        PassTrace* tr) {
  const int n1 = n[1], n2 = n[2];
  const size_t cz = sizeof(V), sz = cz / 2;  // complex and real element sizes
  Jobs j2{}, j3{}, j4{};
  j2.count = j3.count = j4.count = m;
  for (int i = 0; i < m; ++i) {
    const int k = b + i;
    char* Xs = (char*)X[k] + (size_t)k0s * n1 * n2 * cz;
    char* Ys = (char*)Y[k] + (size_t)k0s * n1 * 2 * n2 * cz;
    const char* Ss = (const char*)S[k] + (size_t)k0s * (n1 + 1) * (n2 + 1) * (std::is_same<V, cdw>::value ? 8 : sz);
    j2.j[i] = Job{Xs, Ys, nullptr};
    j3.j[i] = Job{Ys, Ys, Ss};
    j4.j[i] = Job{Ys, Xs, nullptr};
  }
  const long long rows = (long long)pc * n1;
  cudaError_t e = f2.rowf(j2, rows, s);
  if (e == cudaSuccess) e = trace_mark(tr, kRowFwd, s);
  if (e == cudaSuccess) e = f3.colm(j3, 2 * n2, pc, s);
  if (e == cudaSuccess) e = trace_mark(tr, kColMid, s);
  if (e == cudaSuccess) e = f4.rowi(j4, rows, s);
  if (e == cudaSuccess) e = trace_mark(tr, kRowInv, s);
  return e;
}

// The fused outer pair for a grid (0: the separate passes): FP32, n0 = n2.
template <typename V> int fused_pair(const int* n, int dir) {
  if constexpr (!std::is_same<V, float2>::value) {
    return 0;
  } else {
    if (n[0] != n[2]) return 0;
    return fused_config(2 * n[0], dir);
  }
}

template <typename V>
cudaError_t group_passes(const int* n, int count, const void* const* rho, void* const* phi, void* const* X,
                         void* const* Y, const void* const* S, cudaStream_t s, PassTrace* tr,
                         long long chunk_bytes) {
  const int n0 = n[0], n1 = n[1], n2 = n[2];
  const long long C = (long long)n1 * n2;
  const long long rows = (long long)(n0 + 1) * n1;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < count && e == cudaSuccess; b += kMaxJobs) {
    const int m = count - b < kMaxJobs ? count - b : kMaxJobs;
    Jobs j1{}, j2{}, j3{}, j4{}, j5{};
    j1.count = j2.count = j3.count = j4.count = j5.count = m;
    for (int i = 0; i < m; ++i) {
      const int k = b + i;
      j1.j[i] = Job{rho[k], X[k], nullptr};
      j2.j[i] = Job{X[k], Y[k], nullptr};
      j3.j[i] = Job{Y[k], Y[k], S[k]};
      j4.j[i] = Job{Y[k], X[k], nullptr};
      j5.j[i] = Job{X[k], phi[k], nullptr};
    }
    if (e == cudaSuccess) e = trace_mark(tr, -1, s);
    const PassFns& f1 = pass_fns(arith_for<V>(kR2C, 2 * n0), 2 * n0);
    const PassFns& f2 = pass_fns(arith_for<V>(kRowFwd, 2 * n2), 2 * n2);
    const PassFns& f3 = pass_fns(arith_for<V>(kColMid, 2 * n1), 2 * n1);
    const PassFns& f4 = pass_fns(arith_for<V>(kRowInv, 2 * n2), 2 * n2);
    const PassFns& f5 = pass_fns(arith_for<V>(kC2R, 2 * n0), 2 * n0);
    if (!f1.r2c || !f2.rowf || !f3.colm || !f4.rowi || !f5.c2r) return cudaErrorInvalidValue;
    // pass split: slabs of planes whose X + Y fit chunk_bytes stay in L2
    // between the row-forward, middle and row-inverse passes
    const long long plane = (long long)m * n1 * (n2 + 2 * n2) * (long long)sizeof(V);
    const int K0 = n0 + 1;
    int pc = chunk_bytes > 0 ? (int)std::max<long long>(1, chunk_bytes / plane) : K0;
    // the fused outer pairs (rho -> Y, Y -> phi by clusters; no split)
    const int ff = pc >= K0 ? fused_pair<V>(n, 0) : 0;
    const int fi = pc >= K0 ? fused_pair<V>(n, 1) : 0;
    const PassFns& f55 = pass_fns(kArithF32G5, 2 * n0);
    // jobs that share one spectrum (densities of one plan) take the middle
    // pass that reads each spectrum tile once for all of them
    bool shared = m > 1 && f3.colm_shared;
    for (int i = 1; i < m && shared; ++i) shared = j3.j[i].S == j3.j[0].S;
    // the seventh generation: row forward, middle and row inverse as one
    // pipelined kernel (FP32, n1 = n2, not with a fused outer pair)
    const bool pipe = std::is_same<V, float2>::value && pc >= K0 && ff == 0 && fi == 0 && n1 == n2 &&
                      pipe_config(2 * n2) == 1 && pipe_ctr_bytes(n, FSA_F32) > 0;
    if (ff > 0) {
      Jobs jf = j1;
      for (int i = 0; i < m; ++i) jf.j[i].out = Y[b + i];
      e = e == cudaSuccess ? f55.fwd5(ff - 1, jf, n1, s) : e;
      if (e == cudaSuccess) e = trace_mark(tr, kRowFwd, s);
    } else {
      e = e == cudaSuccess ? f1.r2c(j1, C, s) : e;
      if (e == cudaSuccess) e = trace_mark(tr, kR2C, s);
    }
    if (pipe) {
      Jobs jp{};
      jp.count = m;
      const size_t y_bytes = (size_t)K0 * n1 * (2 * (size_t)n2) * sizeof(V);
      for (int i = 0; i < m; ++i)
        jp.j[i] = Job{X[b + i], Y[b + i], S[b + i], i == 0 ? (const void*)((char*)Y[b] + y_bytes) : nullptr};
      if (e == cudaSuccess) e = k7_pipe_fn(2 * n2)(jp, n1, K0, s);
      if (e == cudaSuccess) e = trace_mark(tr, kColMid, s);
    } else if (pc >= K0) {
      if (ff == 0) {
        if (e == cudaSuccess) e = f2.rowf(j2, rows, s);
        if (e == cudaSuccess) e = trace_mark(tr, kRowFwd, s);
      }
      if (e == cudaSuccess) e = shared ? f3.colm_shared(j3, 2 * n2, n0 + 1, s) : f3.colm(j3, 2 * n2, n0 + 1, s);
      if (e == cudaSuccess) e = trace_mark(tr, kColMid, s);
      if (fi == 0) {
        if (e == cudaSuccess) e = f4.rowi(j4, rows, s);
        if (e == cudaSuccess) e = trace_mark(tr, kRowInv, s);
      }
    } else {
      for (int k0s = 0; k0s < K0 && e == cudaSuccess; k0s += pc) {
        const int c = std::min(pc, K0 - k0s);
        e = middle_slab<V>(n, m, b, X, Y, S, k0s, c, f2, f3, f4, s, tr);
      }
    }
    if (fi > 0) {
      Jobs ji = j5;
      for (int i = 0; i < m; ++i) ji.j[i].in = Y[b + i];
      if (e == cudaSuccess) e = f55.inv5(fi - 1, ji, n1, s);
      if (e == cudaSuccess) e = trace_mark(tr, kRowInv, s);
    } else {
      if (e == cudaSuccess) e = f5.c2r(j5, C, s);
      if (e == cudaSuccess) e = trace_mark(tr, kC2R, s);
    }
  }
  return e;
}
template cudaError_t group_passes<float2>(const int*, int, const void* const*, void* const*, void* const*,
                                          void* const*, const void* const*, cudaStream_t, PassTrace*, long long);
template cudaError_t group_passes<double2>(const int*, int, const void* const*, void* const*, void* const*,
                                           void* const*, const void* const*, cudaStream_t, PassTrace*, long long);
template cudaError_t group_passes<cdw>(const int*, int, const void* const*, void* const*, void* const*,
                                       void* const*, const void* const*, cudaStream_t, PassTrace*, long long);

// The d = 2 path (Sec. 2.3 with two axes): R2C along axis 0 over the n1
// real columns, the row middle pass (axis 1 forward, multiply, inverse) in
// place on X, C2R along axis 0, all first-generation kernels with narrow
// tiles (a plane is small: more CTAs per solve).  n = (n0, n1, 1); Y unused.
template <typename V> int first_gen_arith() {
  if constexpr (std::is_same<V, float2>::value) return kArithF32G1;
  else if constexpr (std::is_same<V, double2>::value) return kArithF64;
  else return kArithDW;
}

template <typename V>
cudaError_t group_passes_2d(const int* n, int count, const void* const* rho, void* const* phi, void* const* X,
                            const void* const* S, cudaStream_t s, PassTrace* tr) {
  const int n0 = n[0], n1 = n[1];
  const long long C = n1, rows = n0 + 1;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < count && e == cudaSuccess; b += kMaxJobs) {
    const int m = count - b < kMaxJobs ? count - b : kMaxJobs;
    Jobs j1{}, j2{}, j3{};
    j1.count = j2.count = j3.count = m;
    for (int i = 0; i < m; ++i) {
      const int k = b + i;
      j1.j[i] = Job{rho[k], X[k], nullptr};
      j2.j[i] = Job{X[k], X[k], S[k]};
      j3.j[i] = Job{X[k], phi[k], nullptr};
    }
    const PassFns& f1 = pass_fns(first_gen_arith<V>(), 2 * n0);
    const PassFns& f2 = pass_fns(first_gen_arith<V>(), 2 * n1);
    const PassFns& f3 = f1;
    if (!f1.r2c_plane || !f2.rowm || !f3.c2r_plane) return cudaErrorInvalidValue;
    e = trace_mark(tr, -1, s);
    if (e == cudaSuccess) e = f1.r2c_plane(j1, C, s);
    if (e == cudaSuccess) e = trace_mark(tr, kR2C, s);
    if (e == cudaSuccess) e = f2.rowm(j2, rows, s);
    if (e == cudaSuccess) e = trace_mark(tr, kColMid, s);
    if (e == cudaSuccess) e = f3.c2r_plane(j3, C, s);
    if (e == cudaSuccess) e = trace_mark(tr, kC2R, s);
  }
  return e;
}

// The 3-D DDI (Sec. 5, Example 4) for `count` solves of one plan shape,
// Phi = -(m.n) rho - 3 (1/(4 pi |x|)) * (d_n d_m rho).
// Kernel reading: the five Coulomb passes, the middle one multiplying by
// -3 S D - (m.n)/(8 n0 n1 n2) (par).  Grid reading: -3 d_n d_m rho by five
// passes of the unpadded transform (length n_j per axis; R2C along axis 0
// into Y, row forward Y -> X, middle in place on X with -3 D / (n0 n1 n2),
// row inverse X -> Y, C2R into the back half of Y): the bulk-copy kernels for
// FP32 plans, the first generation in the plan's arithmetic for FP64; then
// the five Coulomb passes on it, the last adding
// -(m.n) rho.  No pass split (the DDI middle pass takes absolute plane
// indices).
size_t align256(size_t b) { return (b + 255) / 256 * 256; }

template <typename V>
cudaError_t group_passes_ddi(const fsa_plan* shape, int count, const void* const* rho, void* const* phi,
                             void* const* X, void* const* Y, const void* const* S, const DdiPar* const* par,
                             cudaStream_t s, PassTrace* tr) {
  using Vu = V;
  const int n0 = shape->n[0], n1 = shape->n[1], n2 = shape->n[2];
  const long long C = (long long)n1 * n2;
  const long long rows = (long long)(n0 + 1) * n1;
  const bool grid = shape->ddi == FSA_DDI_GRID;
  if (!par) return cudaErrorInvalidValue;
  const PassFns& f1 = pass_fns(arith_for<V>(kR2C, 2 * n0), 2 * n0);
  const PassFns& f2 = pass_fns(arith_for<V>(kRowFwd, 2 * n2), 2 * n2);
  const PassFns& f3 = pass_fns(arith_for<V>(kColMid, 2 * n1), 2 * n1);
  const PassFns& f4 = pass_fns(arith_for<V>(kRowInv, 2 * n2), 2 * n2);
  const PassFns& f5 = pass_fns(arith_for<V>(kC2R, 2 * n0), 2 * n0);
  if (!f1.r2c || !f2.rowf || !f3.colm || !f3.colm_ddi || !f4.rowi || !f5.c2r || !f5.c2r_epi)
    return cudaErrorInvalidValue;
  // unpadded passes: the bulk-copy generation for FP32, first generation in
  // the plan's arithmetic for FP64
  const int ua = std::is_same<V, float2>::value ? (int)kArithF32G4 : first_gen_arith<Vu>();
  const PassFns& u0 = pass_fns(ua, n0);
  const PassFns& u1 = pass_fns(ua, n1);
  const PassFns& u2 = pass_fns(ua, n2);
  if (grid && (!u0.r2c_per || !u0.c2r_per || !u1.colm_per || !u2.rowf_per || !u2.rowi_per))
    return cudaErrorInvalidValue;
  const long long Kn = n0 / 2 + 1;  // unpadded half spectrum along axis 0
  const size_t xn_bytes = align256((size_t)Kn * n1 * n2 * sizeof(Vu));
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < count && e == cudaSuccess; b += kMaxJobs) {
    const int m = count - b < kMaxJobs ? count - b : kMaxJobs;
    Jobs g1{}, g2{}, g3{}, g4{}, g5{}, j1{}, j2{}, j3{}, j4{}, j5{};
    g1.count = g2.count = g3.count = g4.count = g5.count = m;
    j1.count = j2.count = j3.count = j4.count = j5.count = m;
    for (int i = 0; i < m; ++i) {
      const int k = b + i;
      char* Yk = static_cast<char*>(Y[k]);
      void* drho = Yk + xn_bytes;
      g1.j[i] = Job{rho[k], Yk, nullptr};
      g2.j[i] = Job{Yk, X[k], nullptr};
      g3.j[i] = Job{X[k], X[k], nullptr, nullptr, par[k]};
      g4.j[i] = Job{X[k], Yk, nullptr};
      g5.j[i] = Job{Yk, drho, nullptr};
      j1.j[i] = Job{grid ? drho : rho[k], X[k], nullptr};
      j2.j[i] = Job{X[k], Y[k], nullptr};
      j3.j[i] = Job{Y[k], Y[k], S[k], nullptr, par[k]};
      j4.j[i] = Job{Y[k], X[k], nullptr};
      j5.j[i] = Job{X[k], phi[k], nullptr, rho[k], par[k]};
    }
    e = trace_mark(tr, -1, s);
    if (grid) {
      if (e == cudaSuccess) e = u0.r2c_per(g1, C, s);
      if (e == cudaSuccess) e = trace_mark(tr, kR2C, s);
      if (e == cudaSuccess) e = u2.rowf_per(g2, Kn * n1, s);
      if (e == cudaSuccess) e = trace_mark(tr, kRowFwd, s);
      if (e == cudaSuccess) e = u1.colm_per(g3, n2, (int)Kn, s);
      if (e == cudaSuccess) e = trace_mark(tr, kColMid, s);
      if (e == cudaSuccess) e = u2.rowi_per(g4, Kn * n1, s);
      if (e == cudaSuccess) e = trace_mark(tr, kRowInv, s);
      if (e == cudaSuccess) e = u0.c2r_per(g5, C, s);
      if (e == cudaSuccess) e = trace_mark(tr, kC2R, s);
    }
    if (e == cudaSuccess) e = f1.r2c(j1, C, s);
    if (e == cudaSuccess) e = trace_mark(tr, kR2C, s);
    if (e == cudaSuccess) e = f2.rowf(j2, rows, s);
    if (e == cudaSuccess) e = trace_mark(tr, kRowFwd, s);
    if (e == cudaSuccess) e = grid ? f3.colm(j3, 2 * n2, n0 + 1, s) : f3.colm_ddi(j3, 2 * n2, n0 + 1, s);
    if (e == cudaSuccess) e = trace_mark(tr, kColMid, s);
    if (e == cudaSuccess) e = f4.rowi(j4, rows, s);
    if (e == cudaSuccess) e = trace_mark(tr, kRowInv, s);
    if (e == cudaSuccess) e = grid ? f5.c2r_epi(j5, C, s) : f5.c2r(j5, C, s);
    if (e == cudaSuccess) e = trace_mark(tr, kC2R, s);
  }
  return e;
}

cudaError_t run_group(const fsa_plan* shape, int count, const void* const* rho, void* const* phi, void* const* X,
                      void* const* Y, const void* const* S, cudaStream_t s, PassTrace* tr,
                      const DdiPar* const* par) {
  if (shape->ddi >= 0) {
    if (shape->dtype == FSA_F32) return group_passes_ddi<float2>(shape, count, rho, phi, X, Y, S, par, s, tr);
    if (shape->f64_dw) return group_passes_ddi<cdw>(shape, count, rho, phi, X, Y, S, par, s, tr);
    return group_passes_ddi<double2>(shape, count, rho, phi, X, Y, S, par, s, tr);
  }
  if (shape->d == 2) {
    if (shape->dtype == FSA_F32) return group_passes_2d<float2>(shape->n, count, rho, phi, X, S, s, tr);
    if (shape->f64_dw) return group_passes_2d<cdw>(shape->n, count, rho, phi, X, S, s, tr);
    return group_passes_2d<double2>(shape->n, count, rho, phi, X, S, s, tr);
  }
  const long long cb = shape->chunk_bytes;
  if (shape->dtype == FSA_F32) return group_passes<float2>(shape->n, count, rho, phi, X, Y, S, s, tr, cb);
  if (shape->f64_dw) return group_passes<cdw>(shape->n, count, rho, phi, X, Y, S, s, tr, cb);
  return group_passes<double2>(shape->n, count, rho, phi, X, Y, S, s, tr, cb);
}

const void* plan_apply_spectrum(const fsa_plan* p) { return p->f64_dw ? p->spectrum_dw : p->spectrum; }

}  // namespace fsa

namespace {

double appendix_b_bound_impl(double R0, double eps);

// The far-field integral for a kernel of Table 1 (see fsa_appendix_b_bound_kernel).

// The Yukawa kernels' far-field integral (fsa_appendix_b_bound_kernel_param):
// int_0^{eps^2/4} f(t) dt with t = (eps^2/4) exp(-y), y in [0, Y], where the
// factor exp(-R0^2/(4t)) = exp(-Q e^y), Q = R0^2/eps^2, has fallen by e^-60;
// 32 panels of the 16-point Gauss-Legendre rule, in long double.
double yukawa_bound(int d, double lam, double R0, double eps) {
  const long double pi = 3.141592653589793238462643383279502884L;
  const long double a = 0.25L * eps * eps, Q = (long double)R0 * R0 / ((long double)eps * eps), L2 = (long double)lam * lam;
  long double gx[16], gw[16];
  gauss_legendre(16, gx, gw);
  const long double Y = logl(1.0L + 60.0L / Q), hw = Y / 64.0L;
  long double sum = 0;
  for (int k = 0; k < 32; ++k) {
    const long double mid = (2 * k + 1) * hw;
    for (int i = 0; i < 16; ++i) {
      const long double y = mid + hw * gx[i], t = a * expl(-y);
      long double f;
      if (d == 2) {
        f = expl(-L2 * t - (long double)R0 * R0 / (4 * t)) / (2 * pi);
      } else {
        f = expl(-L2 * t) * powl(4 * pi * t, -1.5L) *
            (2 * t * R0 * expl(-(long double)R0 * R0 / (4 * t)) + 2 * sqrtl(pi) * powl(t, 1.5L) * erfcl(R0 / (2 * sqrtl(t))));
      }
      sum += gw[i] * hw * f * t;  // dt = t dy
    }
  }
  return (double)sum;
}

double appendix_b_bound_kernel_impl(fsa_kernel kernel, double R0, double eps, double param = 0.0) {
  if (kernel == FSA_KERNEL_YUKAWA3D || kernel == FSA_KERNEL_YUKAWA2D)
    return param > 0 ? yukawa_bound(kernel_dim(kernel), param, R0, eps) : NAN;
  if (kernel == FSA_KERNEL_COULOMB3D) return appendix_b_bound_impl(R0, eps);
  const long double c = (long double)R0 / (long double)eps, e = eps;
  const long double pi = 3.141592653589793238462643383279502884L;
  // d = 2: int_{R0}^inf |U - U^eps| r dr, a = c^2:
  //   Coulomb    (eps/(2 pi)) int_c^inf erfc(s) ds = (eps/(2 pi)) (exp(-c^2)/sqrt(pi) - c erfc(c))
  //   Poisson    (eps^2/(8 pi)) int_a^inf E1(u) du = (eps^2/(8 pi)) (exp(-a) - a E1(a))
  //   biharmonic (eps^4/(32 pi)) int_a^inf u E1(u) du = (eps^4/(64 pi)) ((1 + a) exp(-a) - a^2 E1(a))
  if (kernel == FSA_KERNEL_COULOMB2D) return (double)(e / (2 * pi) * (expl(-c * c) / sqrtl(pi) - c * erfcl(c)));
  if (kernel == FSA_KERNEL_POISSON2D) {
    const long double a = c * c;
    return (double)(e * e / (8 * pi) * (expl(-a) - a * fsa::expint_e1(a)));
  }
  if (kernel == FSA_KERNEL_BIHARMONIC2D) {
    const long double a = c * c;
    return (double)(e * e * e * e / (64 * pi) * ((1 + a) * expl(-a) - a * a * fsa::expint_e1(a)));
  }
  if (kernel != FSA_KERNEL_BIHARMONIC3D) return NAN;
  // (eps^4/(8 pi)) int_c^inf s^3 erfc(s) ds; by parts,
  // int_c^inf s^3 erfc(s) ds = erfc(c) (3/16 - c^4/4) + exp(-c^2) (c^3/2 + 3c/4) / (2 sqrt(pi))
  const long double e4 = (long double)eps * eps * eps * eps;
  const long double tail =
      erfcl(c) * (3.0L / 16.0L - c * c * c * c / 4.0L) + expl(-c * c) * (c * c * c / 2.0L + 0.75L * c) / (2.0L * sqrtl(pi));
  return (double)(e4 * tail / (8.0L * pi));
}

double appendix_b_bound_impl(double R0, double eps) {
  // R0^2 f(c), f(c) = (1/(4 pi c^2)) int_c^inf s erfc(s) ds, c = R0/eps (App. B);
  // int_c^inf s erfc(s) ds = (1/4 - c^2/2) erfc(c) + c exp(-c^2) / (2 sqrt(pi)).
  const long double c = (long double)R0 / (long double)eps;
  const long double pi = 3.141592653589793238462643383279502884L;
  const long double tail = (0.25L - 0.5L * c * c) * erfcl(c) + c * expl(-c * c) / (2.0L * sqrtl(pi));
  return (double)((long double)R0 * R0 * tail / (4.0L * pi * c * c));
}

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  cudaError_t set(int dev) {
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev != prev) {
      e = cudaSetDevice(dev);
      changed = (e == cudaSuccess);
    }
    return e;
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

// unpadded: also the transform lengths n_j themselves (the DDI grid
// reading's unpadded passes)
fsa_status prepare_device(int dev, fsa_dtype dt, const int* n, int d, bool unpadded = false) {
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (!g_tw_ready.count(dev)) {
    cudaError_t e = init_all_twiddles();
    if (e == cudaSuccess) e = tensorgen_init_twiddles();
    if (e != cudaSuccess) return cuda_error(e, "twiddle table upload");
    e = ensure_fault_word_locked(dev);
    if (e != cudaSuccess) return cuda_error(e, "fault word");
    // fsa_apply_noalloc's static scratch: reserved now, while plans are being
    // made, so that the allocation-free apply finds it held.  Not fatal here:
    // that entry point retries the lookup and reports its own error.
    if (noalloc_resolve(dev) != cudaSuccess) cudaGetLastError();
    g_tw_ready.insert(dev);
  }
  for (int jj = 0; jj < (unpadded ? 2 * d : d); ++jj) {  // a plane's unit third axis has no kernels
    const int j = jj % d;
    const int M = jj < d ? 2 * n[j] : n[j];
    const int key = M * 4 + (int)dt;
    if (g_prepared.count({dev, key})) continue;
    cudaError_t e = cudaSuccess;
    const int f32a[5] = {kArithF32G1, kArithF32G2, kArithF32G3, kArithF32G4, kArithF32G6};
    const int f64a[5] = {kArithF64, kArithDW, kArithDW, kArithDW, kArithDW};
    for (int a : (dt == FSA_F32 ? f32a : f64a)) {
      const PassFns& f = pass_fns(a, M);
      if (!f.prepare) return set_error(FSA_ERR_UNSUPPORTED, "no kernels registered for this length");
      if (e == cudaSuccess) e = f.prepare();
    }
    const PassFns& f5g = pass_fns(kArithF32G5, M);  // fused outer pairs (some lengths)
    if (dt == FSA_F32 && f5g.prepare && e == cudaSuccess) e = f5g.prepare();
    if (dt == FSA_F32 && e == cudaSuccess) e = k6_prepare(M);  // the sixth-generation middle pass
    if (dt == FSA_F32 && e == cudaSuccess) e = k8_prepare(M);  // the eighth-generation middle pass
    if (dt == FSA_F32 && e == cudaSuccess) e = k7_prepare(M);  // the seventh-generation pipelined kernel
    if (e == cudaSuccess) e = tensorgen_prepare(M);
    if (e != cudaSuccess) return cuda_error(e, "kernel shared-memory opt-in");
    g_prepared.insert({dev, key});
  }
  return FSA_OK;
}

cudaError_t apply_passes(const fsa_plan* p, const void* rho, void* phi, void* X, void* Y, cudaStream_t s) {
  const void* rhos[1] = {rho};
  void* phis[1] = {phi};
  void* xs[1] = {X};
  void* ys[1] = {Y};
  const void* ss[1] = {plan_apply_spectrum(p)};
  const DdiPar* pars[1] = {p->ddi_par};
  return run_group(p, 1, rhos, phis, xs, ys, ss, s, nullptr, pars);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

namespace fsa {
// All five passes of one plan on one stream.
cudaError_t plan_apply_passes(const fsa_plan* p, const void* rho, void* phi, cudaStream_t s) {
  void* X = p->ws;
  void* Y = (char*)p->ws + p->x_bytes;
  return apply_passes(p, rho, phi, X, Y, s);
}

// The same with a per-launch event trace.
cudaError_t plan_apply_passes_trace(const fsa_plan* p, const void* rho, void* phi, cudaStream_t s,
                                    PassTrace* tr) {
  const void* rhos[1] = {rho};
  void* phis[1] = {phi};
  void* xs[1] = {p->ws};
  void* ys[1] = {(char*)p->ws + p->x_bytes};
  const void* ss[1] = {plan_apply_spectrum(p)};
  const DdiPar* pars[1] = {p->ddi_par};
  return run_group(p, 1, rhos, phis, xs, ys, ss, s, tr, pars);
}
}  // namespace fsa

extern "C" {

const char* fsa_status_string(fsa_status s) {
  switch (s) {
    case FSA_OK: return "FSA_OK";
    case FSA_ERR_INVALID_ARG: return "FSA_ERR_INVALID_ARG";
    case FSA_ERR_UNSUPPORTED: return "FSA_ERR_UNSUPPORTED";
    case FSA_ERR_EPS: return "FSA_ERR_EPS";
    case FSA_ERR_OOM: return "FSA_ERR_OOM";
    case FSA_ERR_CUDA: return "FSA_ERR_CUDA";
    case FSA_ERR_NOT_GENERATED: return "FSA_ERR_NOT_GENERATED";
    case FSA_ERR_BUSY: return "FSA_ERR_BUSY";
    case FSA_ERR_TIMEOUT: return "FSA_ERR_TIMEOUT";
    case FSA_ERR_DEVICE_TIMEOUT: return "FSA_ERR_DEVICE_TIMEOUT";
    case FSA_ERR_NOT_FOUND: return "FSA_ERR_NOT_FOUND";
  }
  return "FSA_ERR_UNKNOWN";
}

const char* fsa_last_error(void) { return t_last_error.c_str(); }

fsa_status fsa_device_fault(int device, unsigned int* code, int clear) {
  if (!code) return set_error(FSA_ERR_INVALID_ARG, "fsa_device_fault: NULL code");
  *code = 0;
  if (device < 0) {
    if (cudaGetDevice(&device) != cudaSuccess) return set_error(FSA_ERR_CUDA, "fsa_device_fault: no device");
  }
  unsigned int* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (device < kMaxDevices) w = g_fault[device];
  }
  if (!w) return FSA_OK;  // nothing ran on this device yet
  DeviceGuard dg;
  cudaError_t e = dg.set(device);
  if (e == cudaSuccess) e = cudaMemcpy(code, w, sizeof(unsigned int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear && *code) e = cudaMemset(w, 0, sizeof(unsigned int));
  if (e != cudaSuccess) return cuda_error(e, "fsa_device_fault");
  return FSA_OK;
}

fsa_status fsa_autotune_set(int mode) {
  if (mode < 0 || mode > 7) return set_error(FSA_ERR_INVALID_ARG, "fsa_autotune_set: mode must be 0..7");
  autotune_mode() = mode;
  apply_graphs_invalidate();
  return FSA_OK;
}

int fsa_fused_configs(int M, int* cluster_ctas, int* threads, int cap) {
  if (M < 0 || M > 1024) return 0;
  const PassFns& f = pass_fns(kArithF32G5, M);
  for (int k = 0; k < f.nfused && k < cap; ++k) {
    if (cluster_ctas) cluster_ctas[k] = f.fused_cs[k];
    if (threads) threads[k] = f.fused_nt[k];
  }
  return f.nfused;
}

fsa_status fsa_pipe_select(int M, int c) {
  if (M < 0 || M > 1024 || !k7_pipe_fn(M))
    return set_error(FSA_ERR_INVALID_ARG, "fsa_pipe_select: no pipelined kernel for this length");
  if (c < -1 || c > 1) return set_error(FSA_ERR_INVALID_ARG, "fsa_pipe_select: c must be -1, 0 or 1");
  set_pipe_config(M, c);
  apply_graphs_invalidate();
  return FSA_OK;
}

fsa_status fsa_fused_select(int M, int dir, int c) {
  const int nf = (M >= 0 && M <= 1024) ? pass_fns(kArithF32G5, M).nfused : 0;
  if (nf == 0) return set_error(FSA_ERR_INVALID_ARG, "fsa_fused_select: no fused configurations for this length");
  if (dir < 0 || dir > 2) return set_error(FSA_ERR_INVALID_ARG, "fsa_fused_select: dir must be 0, 1 or 2");
  if (c < -1 || c > nf) return set_error(FSA_ERR_INVALID_ARG, "fsa_fused_select: configuration out of range");
  for (int d = 0; d < 2; ++d)
    if (dir == 2 || dir == d) set_fused_config(M, d, c);
  apply_graphs_invalidate();
  return FSA_OK;
}

double fsa_appendix_b_bound(double R0, double eps) {
  if (!(R0 > 0) || !(eps > 0)) return NAN;
  return appendix_b_bound_impl(R0, eps);
}

double fsa_appendix_b_bound_kernel(fsa_kernel kernel, double R0, double eps) {
  if (!(R0 > 0) || !(eps > 0)) return NAN;
  return appendix_b_bound_kernel_impl(kernel, R0, eps);
}

double fsa_appendix_b_bound_kernel_param(fsa_kernel kernel, double param, double R0, double eps) {
  if (!(R0 > 0) || !(eps > 0)) return NAN;
  return appendix_b_bound_kernel_impl(kernel, R0, eps, param);
}

}  // extern "C"

namespace fsa {

size_t pipe_ctr_bytes(const int* n, fsa_dtype dt) {
  if (dt != FSA_F32 || n[2] < 2 || n[1] != n[2] || !k7_pipe_fn(2 * n[2])) return 0;
  return align256(sizeof(unsigned) * (2 + 2 * (size_t)(n[0] + 1) * kMaxJobs));
}

size_t plan_workspace_bytes(const int* n, fsa_dtype dt) {
  const size_t s = dt == FSA_F32 ? 4 : 8;
  const size_t K0 = n[0] + 1;
  return K0 * n[1] * n[2] * 2 * s + K0 * n[1] * (2 * (size_t)n[2]) * 2 * s + pipe_ctr_bytes(n, dt);
}

// Reals in the spectrum octant: (n0+1)(n1+1)(n2+1), or (n0+1)(n1+1) for a
// plane (held with n[2] = 1).
static size_t octant_count(const int* n, int d) {
  return (size_t)(n[0] + 1) * (n[1] + 1) * (d == 2 ? 1 : n[2] + 1);
}

// FP32 plans generate in FP64 in a scratch octant; FP64 plans in place.
size_t plan_gen_scratch_bytes(const int* n, fsa_dtype dt, int d) {
  return dt == FSA_F64 ? 0 : octant_count(n, d) * 8;
}

// Device bytes a plan without workspace holds: the spectrum octant in its
// dtype, and for FP64 plans the double-word copy of it (same size).
size_t plan_resident_bytes(const int* n, fsa_dtype dt, int d) {
  const size_t s = dt == FSA_F32 ? 4 : 8;
  return octant_count(n, d) * s * (dt == FSA_F64 ? 2 : 1);
}

cudaError_t tune_plan(fsa_plan* p);

// Argument checks that need no device.  On success *eps_out / *bound_out
// hold the eps in use and its App. B bound.
fsa_status plan_validate(fsa_kernel kernel, const double* L, const int* n, fsa_dtype dtype, double eps_in,
                         double eps_tol, double* eps_out, double* bound_out, double param = 0.0) {
  if (kernel < FSA_KERNEL_COULOMB3D || kernel > FSA_KERNEL_YUKAWA2D || kernel == FSA_KERNEL_DDI3D)
    return set_error(FSA_ERR_UNSUPPORTED, "fsa_plan_create: unknown kernel");
  if (dtype != FSA_F32 && dtype != FSA_F64) return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create: bad dtype");
  const int d = kernel_dim(kernel);
  for (int j = 0; j < d; ++j) {
    if (!supported_n(n[j]))
      return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create: n[" + std::to_string(j) + "] = " +
                                                std::to_string(n[j]) +
                                                " unsupported (need even 2^a or 3*2^a in [4, 512])");
    if (!(L[j] > 0) || !std::isfinite(L[j]))
      return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create: L[" + std::to_string(j) + "] must be > 0");
  }
  if (eps_in < 0 || !std::isfinite(eps_in)) return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create: eps < 0");
  const double R0 = 2.0 * (d == 2 ? std::min(L[0], L[1]) : std::min(L[0], std::min(L[1], L[2])));
  const double eps = eps_in > 0 ? eps_in : std::min(1.0, R0 / 6.0);
  const double bound = appendix_b_bound_kernel_impl(kernel, R0, eps, param);
  // Default tolerance: App. B's eps_tol = 1e-16 (16 digits) for FP64 plans,
  // so that an FP64 solve cannot carry a far-field truncation far above its
  // round-off; 1e-8 for FP32 plans (round-off near 1e-7).
  const double tol = eps_tol == 0 ? (dtype == FSA_F64 ? 1e-16 : 1e-8) : eps_tol;
  if (tol > 0 && !(bound <= tol)) {
    char buf[256];
    snprintf(buf, sizeof buf, "fsa_plan_create: eps = %g fails App. B: int_R0^inf |U - U^eps| r^2 dr = %.3g > %.3g (R0 = %g)",
             eps, bound, tol, R0);
    return set_error(FSA_ERR_EPS, buf);
  }
  *eps_out = eps;
  *bound_out = bound;
  return FSA_OK;
}

// extra_ws: device bytes appended to the workspace; unpadded: prepare the
// kernels of the transform lengths n_j too (the DDI grid reading).
fsa_status plan_create_core(fsa_plan** out, fsa_kernel kernel, const double* L, const int* n, fsa_dtype dtype,
                            double eps_in, double eps_tol, bool with_workspace, size_t extra_ws, bool unpadded,
                            double param = 0.0) {
  *out = nullptr;
  double eps = 0, bound = 0;
  fsa_status vs = plan_validate(kernel, L, n, dtype, eps_in, eps_tol, &eps, &bound, param);
  if (vs != FSA_OK) return vs;
  const int d = kernel_dim(kernel);
  const double R0 = 2.0 * (d == 2 ? std::min(L[0], L[1]) : std::min(L[0], std::min(L[1], L[2])));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "fsa_plan_create: cudaGetDevice");
  fsa_status st = prepare_device(dev, dtype, n, d, unpadded);
  if (st != FSA_OK) return st;

  fsa_plan* p = new fsa_plan{};
  for (int j = 0; j < 3; ++j) {
    p->n[j] = n[j];
    p->L[j] = L[j];
    p->h[j] = 2.0 * L[j] / n[j];
  }
  p->eps = eps;
  p->R0 = R0;
  p->eps_bound = bound;
  p->kernel = kernel;
  p->param = param;
  p->d = d;
  p->ddi = -1;
  p->many_cap = 1;
  p->chunk_bytes = 0;  // one slab: measured fastest at 256^3 (see fsa_plan_opts.l2_chunk_mb)
  p->dtype = dtype;
  p->device = dev;
  const size_t s = dtype == FSA_F32 ? 4 : 8;
  p->spectrum_bytes = octant_count(n, d) * s;
  p->x_bytes = (size_t)(n[0] + 1) * n[1] * n[2] * 2 * s;
  p->ws_bytes = with_workspace ? plan_workspace_bytes(n, dtype) + extra_ws : 0;
  // The workspace always holds the FP64 generation scratch of an FP32 plan.
  e = cudaMalloc(&p->spectrum, p->spectrum_bytes);
  if (e == cudaSuccess && dtype == FSA_F64) e = cudaMalloc(&p->spectrum_dw, p->spectrum_bytes);
  if (e == cudaSuccess && with_workspace) e = cudaMalloc(&p->ws, p->ws_bytes);
  if (e != cudaSuccess) {
    if (p->spectrum) cudaFree(p->spectrum);
    if (p->spectrum_dw) cudaFree(p->spectrum_dw);
    delete p;
    cudaGetLastError();
    return cuda_error(e, "fsa_plan_create: cudaMalloc");
  }
  e = tune_plan(p);
  if (e != cudaSuccess) {
    cudaFree(p->spectrum);
    if (p->spectrum_dw) cudaFree(p->spectrum_dw);
    if (p->ws) cudaFree(p->ws);
    delete p;
    cudaGetLastError();
    return cuda_error(e, "fsa_plan_create: autotune");
  }
  *out = p;
  return FSA_OK;
}

fsa_status plan_create_internal(fsa_plan** out, fsa_kernel kernel, const double* L, const int* n, fsa_dtype dtype,
                                double eps_in, double eps_tol, bool with_workspace, double param) {
  return plan_create_core(out, kernel, L, n, dtype, eps_in, eps_tol, with_workspace, 0, false, param);
}

// The DDI parameter block (fsa_consts.h) of a plan: transform lengths
// M_j = 2 n_j for the kernel reading (the doubled grid, period 4 L_j) and
// n_j for the grid reading (period 2 L_j).
void ddi_params(const fsa_plan* p, int derivative, DdiPar* block) {
  double* par = block->d;
  const double pi = 3.141592653589793238462643383279502884;
  const bool grid = derivative == FSA_DDI_GRID;
  double nm = 0;
  for (int j = 0; j < 3; ++j) {
    const double M = grid ? p->n[j] : 2.0 * p->n[j];
    par[kDdiN + j] = p->dipole_n[j];
    par[kDdiM + j] = p->dipole_m[j];
    par[kDdiW + j] = 2.0 * pi / (M * p->h[j]);
    par[kDdiNu + j] = -pi / p->h[j];
    nm += p->dipole_n[j] * p->dipole_m[j];
  }
  const double vol = (double)p->n[0] * p->n[1] * p->n[2];
  par[kDdiCmul] = grid ? -3.0 / vol : -3.0;
  par[kDdiCadd] = grid ? 0.0 : -nm / (8.0 * vol);
  par[kDdiNyq0] = grid ? p->n[0] / 2 : p->n[0];
  par[kDdiBeta] = -nm;
  par[kDdiC2] = -par[kDdiCmul] * par[kDdiN + 1] * par[kDdiM + 1] * par[kDdiW + 1] * par[kDdiW + 1];
  for (int i = 0; i < kDdiParCount; ++i) {
    block->f[i] = (float)par[i];
    block->lo[i] = (float)(par[i] - (double)block->f[i]);
  }
  block->nyq0 = grid ? p->n[0] / 2 : p->n[0];
}

// The per-line coefficients (c0, c1, cN) of the DDI middle pass (fsa_consts.h)
// for k0 in [0, nyq0], k2 in [0, M2), computed in FP64 and stored in the
// plan's arithmetic: 3 floats (FP32), 3 doubles (native FP64) or 3
// double-word float pairs.  Returns the bytes written to out (null: size only).
size_t ddi_table(const fsa_plan* p, const DdiPar& b, void* out) {
  const double* par = b.d;
  const bool grid = p->ddi == FSA_DDI_GRID;
  const int K0 = b.nyq0 + 1, M2 = grid ? p->n[2] : 2 * p->n[2];
  const int kind = p->dtype == FSA_F32 ? 0 : (p->f64_dw ? 2 : 1);
  const size_t each = kind == 0 ? 12 : 24;
  const size_t bytes = (size_t)K0 * M2 * each;
  if (!out) return bytes;
  const double cm = par[kDdiCmul], n1 = par[kDdiN + 1], m1 = par[kDdiM + 1];
  const double w1 = par[kDdiW + 1], nu1 = par[kDdiNu + 1];
  for (int k0 = 0; k0 < K0; ++k0) {
    const bool y0 = k0 == b.nyq0;
    const double mu0 = y0 ? 0.0 : k0 * par[kDdiW + 0], nu0 = y0 ? par[kDdiNu + 0] : 0.0;
    for (int k2 = 0; k2 < M2; ++k2) {
      const bool y2 = k2 == M2 / 2;
      const double mu2 = y2 ? 0.0 : (k2 < M2 / 2 ? k2 : k2 - M2) * par[kDdiW + 2];
      const double nu2 = y2 ? par[kDdiNu + 2] : 0.0;
      const double a = par[kDdiN] * mu0 + par[kDdiN + 2] * mu2, bb = par[kDdiM] * mu0 + par[kDdiM + 2] * mu2;
      const double an = par[kDdiN] * nu0 + par[kDdiN + 2] * nu2, bn = par[kDdiM] * nu0 + par[kDdiM + 2] * nu2;
      const double c[3] = {-cm * (a * bb + an * bn), -cm * (a * m1 + bb * n1) * w1,
                           -cm * (a * bb + (an + n1 * nu1) * (bn + m1 * nu1))};
      const size_t i = (size_t)k0 * M2 + k2;
      for (int j = 0; j < 3; ++j) {
        if (kind == 0) {
          static_cast<float*>(out)[3 * i + j] = (float)c[j];
        } else if (kind == 1) {
          static_cast<double*>(out)[3 * i + j] = c[j];
        } else {
          const float hi = (float)c[j];
          static_cast<float*>(out)[6 * i + 2 * j] = hi;
          static_cast<float*>(out)[6 * i + 2 * j + 1] = (float)(c[j] - (double)hi);
        }
      }
    }
  }
  return bytes;
}

// Autotuner: for an FP32 plan, time both kernel generations of each pass on the
// plan's own workspace (contents irrelevant: the kernels' cost does not depend
// on the data) and keep the faster for that pass and length.
cudaError_t tune_f64(fsa_plan* p);

cudaError_t tune_plan(fsa_plan* p) {
  if (p->dtype == FSA_F64) return tune_f64(p);
  if (!p->ws || autotune_mode() != 1 || p->d == 2) return cudaSuccess;  // d = 2: defaults
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const int n0 = p->n[0], n1 = p->n[1], n2 = p->n[2];
  const int Ms[kNumPass] = {2 * n0, 2 * n2, 2 * n1, 2 * n2, 2 * n0};
  bool need = false;
  for (int k = 0; k < kNumPass; ++k) need |= g_variant[k][Ms[k]][FSA_F32].load() == 0;
  const PassFns& f5g = pass_fns(kArithF32G5, 2 * n0);
  fused_table_init();
  const bool fuse = n0 == n2 && f5g.nfused > 0;
  for (int dir = 0; dir < 2 && fuse; ++dir) need |= g_fused[2 * n0][dir].load() < 0;
  if (!need) return cudaSuccess;
  cudaStream_t s;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  void* X = p->ws;
  void* Y = (char*)p->ws + p->x_bytes;
  const long long C = (long long)n1 * n2, rows = (long long)(n0 + 1) * n1;
  Jobs j{};
  j.count = 1;
  auto run = [&](int k, int v) -> cudaError_t {
    const PassFns& f = pass_fns(arith_of_variant(v), Ms[k]);
    switch (k) {
      case kR2C: j.j[0] = Job{Y, X, nullptr}; return f.r2c(j, C, s);
      case kRowFwd: j.j[0] = Job{X, Y, nullptr}; return f.rowf(j, rows, s);
      case kColMid: j.j[0] = Job{Y, Y, p->spectrum}; return f.colm(j, 2 * n2, n0 + 1, s);
      case kRowInv: j.j[0] = Job{Y, X, nullptr}; return f.rowi(j, rows, s);
      default: j.j[0] = Job{X, Y, nullptr}; return f.c2r(j, C, s);
    }
  };
  // a short burst first, so that the SM clock has left its idle level before
  // anything is timed
  for (int rep = 0; rep < 20 && e == cudaSuccess; ++rep) e = run(kColMid, 2);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (int k = 0; k < kNumPass && e == cudaSuccess; ++k) {
    if (g_variant[k][Ms[k]][FSA_F32].load() != 0) continue;
    // variants 5 and 6 (the sixth-generation middle pass, the
    // eighth-generation middle, R2C and C2R passes) only where they exist
    std::vector<int> cand = {1, 2, 3, 4};
    if (k == kColMid && k6_colm(Ms[k])) cand.push_back(5);
    if ((k == kColMid && k8_colm(Ms[k])) || (k == kR2C && k8_r2c(Ms[k])) || (k == kC2R && k8_c2r(Ms[k])))
      cand.push_back(6);
    float tmin[7] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
    for (int v : cand) {
      if (e == cudaSuccess) e = run(k, v);  // warm-up
    }
    // rounds over all variants (not one variant after another), so that a
    // drifting clock or a neighbour's load touches every variant alike; the
    // best of five rounds per variant
    for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
      for (int v : cand) {
        if (e != cudaSuccess) break;
        cudaEventRecord(e0, s);
        e = run(k, v);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        tmin[v] = std::min(tmin[v], ms);
      }
    }
    int pick = 2;
    for (int v : cand)
      if (tmin[v] < tmin[pick]) pick = v;
    set_kernel_variant(k, Ms[k], FSA_F32, e == cudaSuccess ? pick : 0);
  }
  // the fused outer pairs against the separate passes just chosen (X stands
  // in for rho and phi: the kernels' cost does not depend on the data)
  auto run_pair = [&](int dir, int c) -> cudaError_t {
    if (c == 0) {
      const int a = dir == 0 ? kR2C : kRowInv, b = dir == 0 ? kRowFwd : kC2R;
      cudaError_t r = run(a, kernel_variant(a, Ms[a], FSA_F32));
      return r == cudaSuccess ? run(b, kernel_variant(b, Ms[b], FSA_F32)) : r;
    }
    j.j[0] = dir == 0 ? Job{X, Y, nullptr} : Job{Y, X, nullptr};
    return dir == 0 ? f5g.fwd5(c - 1, j, n1, s) : f5g.inv5(c - 1, j, n1, s);
  };
  for (int dir = 0; dir < 2 && fuse && e == cudaSuccess; ++dir) {
    if (g_fused[2 * n0][dir].load() >= 0) continue;
    float best = 1e30f;
    int pick = 0;
    for (int c = 0; c <= f5g.nfused && e == cudaSuccess; ++c) {
      e = run_pair(dir, c);  // warm-up
      if (c > 0 && (e == cudaErrorInvalidConfiguration || e == cudaErrorInvalidClusterSize)) {
        // a cluster configuration this device cannot place: not a candidate
        cudaGetLastError();
        e = cudaSuccess;
        continue;
      }
      float tmin = 1e30f;
      for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        e = run_pair(dir, c);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        tmin = std::min(tmin, ms);
      }
      if (tmin < best) {
        best = tmin;
        pick = c;
      }
    }
    if (e == cudaSuccess) set_fused_config(2 * n0, dir, pick);
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  return e;
}

// FP64 plans: native FP64 or double-word arithmetic, one choice per grid
// shape for the whole process (every plan of a shape computes alike, so
// batched and served results equal single ones).  Mode 1 times one whole
// apply each way on the first plan of a shape; mode 0 takes double-word;
// mode 2 / 3 force native / double-word.
cudaError_t tune_f64(fsa_plan* p) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, int> choice;
  const int mode = autotune_mode();
  if (mode >= 2) {
    p->f64_dw = mode >= 3;
    return cudaSuccess;
  }
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(p->n[0], p->n[1], p->n[2]);
  auto it = choice.find(key);
  if (it != choice.end()) {
    p->f64_dw = it->second;
    return cudaSuccess;
  }
  if (mode != 1 || !p->ws) {
    p->f64_dw = 1;
    // a plan without workspace (a serving plan) cannot be timed: it takes
    // double-word, and in mode 1 that becomes the shape's choice, so that every
    // later plan of the shape computes alike (served = solved alone)
    if (mode == 1) choice[key] = 1;
    return cudaSuccess;
  }
  cudaStream_t s;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  void* X = p->ws;
  void* Y = (char*)p->ws + p->x_bytes;
  float best[2] = {1e30f, 1e30f};
  for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
    p->f64_dw = v;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0, s);
      e = apply_passes(p, Y, Y, X, Y, s);
      cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best[v] = std::min(best[v], ms);
    }
  }
  p->f64_dw = best[1] <= best[0] ? 1 : 0;
  if (e == cudaSuccess) choice[key] = p->f64_dw;
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  return e;
}

// fsa_plan_opts.w_quadrature: tabulate W(k) on [0, |mu|_max] by the radial
// Gauss-Kronrod quadrature (radial_w.cpp) and copy the table to the device.
fsa_status attach_w_table(fsa_plan* p) {
  const double pi = 3.141592653589793238462643383279502884;
  double k2 = 0;
  for (int j = 0; j < p->d; ++j) {
    const double m = pi * p->n[j] / (2.0 * p->L[j]);
    k2 += m * m;
  }
  const fsa_kernel k = p->kernel == FSA_KERNEL_DDI3D ? FSA_KERNEL_COULOMB3D : p->kernel;
  std::vector<double> tab;
  int panels = 0;
  if (!radial_w_table(k, p->param, p->eps, std::sqrt(k2), &tab, &panels))
    return set_error(FSA_ERR_CUDA, "fsa_plan_create: W quadrature table failed");
  cudaError_t e = cudaMalloc(&p->wtab, tab.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(p->wtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (p->wtab) cudaFree(p->wtab);
    p->wtab = nullptr;
    cudaGetLastError();
    return cuda_error(e, "fsa_plan_create: W table upload");
  }
  p->wtab_panels = panels;
  return FSA_OK;
}

cudaError_t plan_generate_into(fsa_plan* p, void* scratch, cudaStream_t s) {
  double* oct = p->dtype == FSA_F64 ? (double*)p->spectrum : (double*)scratch;
  // a DDI plan's tensor is the Coulomb kernel's (Sec. 5, Example 4)
  const fsa_kernel k = p->kernel == FSA_KERNEL_DDI3D ? FSA_KERNEL_COULOMB3D : p->kernel;
  cudaError_t e = tensorgen_run(k, p->n, p->L, p->eps, p->param, oct, p->spectrum, p->dtype, s, p->wtab,
                                p->wtab_panels);
  if (e == cudaSuccess && p->spectrum_dw)
    e = spectrum_to_dw((const double*)p->spectrum, p->spectrum_dw, p->spectrum_bytes / 8, s);
  if (e == cudaSuccess) p->generated = 1;
  return e;
}

}  // namespace fsa

extern "C" {

fsa_status fsa_plan_create(fsa_plan** out, fsa_kernel kernel, int d, const double* L, const int* n,
                           fsa_dtype dtype, const fsa_plan_opts* opts) {
  if (!out) return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create: out is NULL");
  *out = nullptr;
  if (kernel == FSA_KERNEL_DDI3D)
    return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create: DDI plans need their dipoles: use fsa_plan_create_ddi3d");
  if (kernel < FSA_KERNEL_COULOMB3D || kernel > FSA_KERNEL_YUKAWA2D)
    return set_error(FSA_ERR_UNSUPPORTED, "fsa_plan_create: unknown kernel");
  if (d != kernel_dim(kernel))
    return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create: d = " + std::to_string(d) + " does not match the kernel (d = " +
                                              std::to_string(kernel_dim(kernel)) + ")");
  if (!L || !n) return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create: L or n is NULL");
  // internally every plan has three axes; a plane (d = 2) has n[2] = 1
  const double L3[3] = {L[0], L[1], d == 3 ? L[2] : 1.0};
  const int n3[3] = {n[0], n[1], d == 3 ? n[2] : 1};
  L = L3;
  n = n3;
  fsa_plan_opts o{};
  o.device = -1;
  if (opts) o = *opts;
  if (!(o.kernel_param >= 0) || !std::isfinite(o.kernel_param))
    return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create: kernel_param must be finite and >= 0");
  // the Yukawa lam (0 selects 1); no parameter for the other kernels
  const double param = kernel_has_param(kernel) ? (o.kernel_param > 0 ? o.kernel_param : 1.0) : 0.0;
  double eps = 0, bound = 0;
  fsa_status vs = plan_validate(kernel, L, n, dtype, o.eps, o.eps_tol, &eps, &bound, param);
  if (vs != FSA_OK) return vs;  // no device touched
  DeviceGuard dg;
  cudaError_t e = dg.set(o.device);
  if (e != cudaSuccess) return cuda_error(e, "fsa_plan_create: cudaSetDevice");
  fsa_status st = plan_create_core(out, kernel, L, n, dtype, o.eps, o.eps_tol, true, 0, false, param);
  if (st == FSA_OK && o.l2_chunk_mb != 0) (*out)->chunk_bytes = o.l2_chunk_mb > 0 ? (long long)o.l2_chunk_mb << 20 : 0;
  if (st == FSA_OK && o.w_quadrature == 1) {
    st = attach_w_table(*out);
    if (st != FSA_OK) {
      fsa_plan_destroy(*out);
      *out = nullptr;
    }
  }
  return st;
}

fsa_status fsa_plan_create_ddi3d(fsa_plan** out, const double* L, const int* n, fsa_dtype dtype,
                                 const double* dipole_n, const double* dipole_m, fsa_ddi_derivative derivative,
                                 const fsa_plan_opts* opts) {
  if (!out) return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create_ddi3d: out is NULL");
  *out = nullptr;
  if (!L || !n || !dipole_n || !dipole_m)
    return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create_ddi3d: NULL argument");
  if (derivative != FSA_DDI_GRID && derivative != FSA_DDI_KERNEL)
    return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create_ddi3d: unknown derivative");
  for (int j = 0; j < 3; ++j)
    if (!std::isfinite(dipole_n[j]) || !std::isfinite(dipole_m[j]))
      return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create_ddi3d: dipoles must be finite");
  fsa_plan_opts o{};
  o.device = -1;
  if (opts) o = *opts;
  double eps = 0, bound = 0;
  fsa_status vs = plan_validate(FSA_KERNEL_COULOMB3D, L, n, dtype, o.eps, o.eps_tol, &eps, &bound);
  if (vs != FSA_OK) return vs;  // no device touched
  const bool grid = derivative == FSA_DDI_GRID;
  for (int j = 0; j < 3 && grid; ++j)
    if (n[j] < 8)
      return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_create_ddi3d: the grid reading needs n_j >= 8");
  DeviceGuard dg;
  cudaError_t e = dg.set(o.device);
  if (e != cudaSuccess) return cuda_error(e, "fsa_plan_create_ddi3d: cudaSetDevice");
  const size_t stage = (size_t)n[0] * n[1] * n[2] * (dtype == FSA_F32 ? 4 : 8);
  fsa_plan* p = nullptr;
  fsa_status st = plan_create_core(&p, FSA_KERNEL_COULOMB3D, L, n, dtype, o.eps, o.eps_tol, true, stage + 256, grid);
  if (st != FSA_OK) return st;
  p->kernel = FSA_KERNEL_DDI3D;
  p->ddi = derivative;
  for (int j = 0; j < 3; ++j) {
    p->dipole_n[j] = dipole_n[j];
    p->dipole_m[j] = dipole_m[j];
  }
  if (o.w_quadrature == 1) {
    st = attach_w_table(p);
    if (st != FSA_OK) {
      fsa_plan_destroy(p);
      return st;
    }
  }
  DdiPar par{};
  ddi_params(p, derivative, &par);
  // one allocation: the block, then the per-line coefficient table
  const size_t off = align256(sizeof(DdiPar));
  std::vector<unsigned char> tab(ddi_table(p, par, nullptr));
  ddi_table(p, par, tab.data());
  e = cudaMalloc(&p->ddi_par, off + tab.size());
  if (e == cudaSuccess) {
    par.tab = reinterpret_cast<const unsigned char*>(p->ddi_par) + off;
    e = cudaMemcpy(p->ddi_par, &par, sizeof par, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(reinterpret_cast<unsigned char*>(p->ddi_par) + off, tab.data(), tab.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    fsa_plan_destroy(p);
    cudaGetLastError();
    return cuda_error(e, "fsa_plan_create_ddi3d: parameter block");
  }
  *out = p;
  return FSA_OK;
}

fsa_status fsa_plan_destroy(fsa_plan* p) {
  if (!p) return FSA_OK;
  batched_forget_plan(p);
  apply_graphs_forget_plan(p);
  DeviceGuard dg;
  dg.set(p->device);
  if (p->ddi_par) cudaFree(p->ddi_par);
  if (p->wtab) cudaFree(p->wtab);
  if (p->ws_many) cudaFree(p->ws_many);
  cudaFree(p->spectrum);
  if (p->spectrum_dw) cudaFree(p->spectrum_dw);
  if (p->ws) cudaFree(p->ws);
  delete p;
  return FSA_OK;
}

fsa_status fsa_plan_spectrum_copy(const fsa_plan* p, void* dst, size_t nbytes, fsa_stream_t stream) {
  if (!p || !dst) return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_spectrum_copy: NULL argument");
  if (nbytes < p->spectrum_bytes) return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_spectrum_copy: dst too small");
  DeviceGuard dg;
  cudaError_t e = dg.set(p->device);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst, p->spectrum, p->spectrum_bytes, cudaMemcpyDefault, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "fsa_plan_spectrum_copy");
  return FSA_OK;
}

fsa_status fsa_plan_info_get(const fsa_plan* p, fsa_plan_info* info) {
  if (!p || !info) return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_info_get: NULL argument");
  for (int j = 0; j < 3; ++j) {
    info->n[j] = p->n[j];
    info->L[j] = p->L[j];
    info->h[j] = p->h[j];
  }
  info->eps = p->eps;
  info->R0 = p->R0;
  info->eps_bound = p->eps_bound;
  info->dtype = p->dtype;
  info->device = p->device;
  info->generated = p->generated;
  info->arithmetic = p->dtype == FSA_F32 ? 0 : (p->f64_dw ? 2 : 1);
  {
    const long long cz = p->dtype == FSA_F32 ? 8 : 16;
    const long long plane = (long long)p->n[1] * 3 * p->n[2] * cz;
    const int K0 = p->n[0] + 1;
    const int pc = p->chunk_bytes > 0 ? (int)std::max<long long>(1, p->chunk_bytes / plane) : K0;
    info->launches_per_apply = p->d == 2 ? 3 : 2 + 3 * ((K0 + std::min(pc, K0) - 1) / std::min(pc, K0));
    const bool fusable = p->d == 3 && p->ddi < 0 && pc >= K0 && p->dtype == FSA_F32;
    info->fused_fwd = fusable ? fused_pair<float2>(p->n, 0) : 0;
    info->fused_inv = fusable ? fused_pair<float2>(p->n, 1) : 0;
    info->launches_per_apply -= (info->fused_fwd > 0) + (info->fused_inv > 0);
    info->pipe = fusable && !info->fused_fwd && !info->fused_inv && p->n[1] == p->n[2] &&
                 pipe_config(2 * p->n[2]) == 1 && pipe_ctr_bytes(p->n, FSA_F32) > 0;
    if (info->pipe) info->launches_per_apply = 3;
    if (p->ddi >= 0) info->launches_per_apply = p->ddi == FSA_DDI_GRID ? 10 : 5;
  }
  info->w_quadrature = p->wtab ? 1 : 0;
  info->w_panels = p->wtab_panels;
  info->workspace_bytes = p->ws_bytes;
  info->spectrum_bytes = p->spectrum_bytes;
  info->spectrum = p->spectrum;
  info->kernel = p->kernel;
  info->d = p->d;
  info->kernel_param = p->param;
  info->many_capacity = p->many_cap;
  info->ddi_derivative = p->ddi;
  for (int j = 0; j < 3; ++j) {
    info->dipole_n[j] = p->ddi >= 0 ? p->dipole_n[j] : 0.0;
    info->dipole_m[j] = p->ddi >= 0 ? p->dipole_m[j] : 0.0;
  }
  return FSA_OK;
}

fsa_status fsa_tensor_generate(fsa_plan* p, fsa_stream_t stream) {
  if (!p) return set_error(FSA_ERR_INVALID_ARG, "fsa_tensor_generate: plan is NULL");
  DeviceGuard dg;
  cudaError_t e = dg.set(p->device);
  if (e != cudaSuccess) return cuda_error(e, "fsa_tensor_generate: cudaSetDevice");
  if (!p->ws && p->dtype == FSA_F32)
    return set_error(FSA_ERR_INVALID_ARG, "fsa_tensor_generate: plan has no workspace for its FP64 scratch");
  e = plan_generate_into(p, p->ws, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "fsa_tensor_generate: launch");
  return FSA_OK;
}

fsa_status fsa_apply(const fsa_plan* p, const void* rho, void* phi, fsa_stream_t stream) {
  if (!p || !rho || !phi) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply: NULL argument");
  if (!p->ws) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply: plan has no workspace");
  if (!p->generated) return set_error(FSA_ERR_NOT_GENERATED, "fsa_apply: call fsa_tensor_generate first");
  if (!aligned16(rho) || !aligned16(phi))
    return set_error(FSA_ERR_INVALID_ARG, "fsa_apply: rho and phi must be 16-byte aligned");
  DeviceGuard dg;
  cudaError_t e = dg.set(p->device);
  if (e == cudaSuccess) e = plan_apply_graph(p, rho, phi, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "fsa_apply: launch");
  return FSA_OK;
}

fsa_status fsa_plan_reserve(fsa_plan* p, int count) {
  if (!p || count < 1) return set_error(FSA_ERR_INVALID_ARG, "fsa_plan_reserve: NULL plan or count < 1");
  if (count <= p->many_cap) return FSA_OK;
  DeviceGuard dg;
  cudaError_t e = dg.set(p->device);
  if (e != cudaSuccess) return cuda_error(e, "fsa_plan_reserve: cudaSetDevice");
  const size_t stride = align256(plan_workspace_bytes(p->n, p->dtype));
  void* mem = nullptr;
  e = cudaMalloc(&mem, stride * (size_t)(count - 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(FSA_ERR_OOM, "fsa_plan_reserve: cudaMalloc of " + std::to_string(stride * (count - 1)) + " bytes");
  }
  // the old workspaces may still be in use by queued work: free them in order
  if (p->ws_many) {
    cudaDeviceSynchronize();
    cudaFree(p->ws_many);
  }
  p->ws_many = mem;
  p->many_stride = stride;
  p->many_cap = count;
  return FSA_OK;
}

fsa_status fsa_apply_many(const fsa_plan* p, const void* const* rho, void* const* phi, int count,
                          fsa_stream_t stream) {
  if (!p || !rho || !phi) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_many: NULL argument");
  if (count < 1 || count > p->many_cap)
    return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_many: count " + std::to_string(count) + " outside [1, " +
                                              std::to_string(p->many_cap) + "] (fsa_plan_reserve grows it)");
  if (!p->ws) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_many: plan has no workspace");
  if (!p->generated) return set_error(FSA_ERR_NOT_GENERATED, "fsa_apply_many: call fsa_tensor_generate first");
  std::vector<const void*> r(count), S(count, plan_apply_spectrum(p));
  std::vector<void*> f(count), X(count), Y(count);
  std::vector<const DdiPar*> par(count, p->ddi_par);
  for (int k = 0; k < count; ++k) {
    if (!rho[k] || !phi[k] || !aligned16(rho[k]) || !aligned16(phi[k]))
      return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_many: rho and phi must be non-NULL and 16-byte aligned");
    r[k] = rho[k];
    f[k] = phi[k];
    X[k] = k == 0 ? p->ws : static_cast<char*>(p->ws_many) + (size_t)(k - 1) * p->many_stride;
    Y[k] = static_cast<char*>(X[k]) + p->x_bytes;
  }
  DeviceGuard dg;
  cudaError_t e = dg.set(p->device);
  if (e == cudaSuccess)
    e = run_group(p, count, r.data(), f.data(), X.data(), Y.data(), S.data(), (cudaStream_t)stream, nullptr,
                  par.data());
  if (e != cudaSuccess) return cuda_error(e, "fsa_apply_many: launch");
  return FSA_OK;
}

fsa_status fsa_apply_host(const fsa_plan* p, const void* rho_host, void* phi_host, fsa_stream_t stream) {
  if (!p || !rho_host || !phi_host) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_host: NULL argument");
  if (!p->ws) return set_error(FSA_ERR_INVALID_ARG, "fsa_apply_host: plan has no workspace");
  if (!p->generated) return set_error(FSA_ERR_NOT_GENERATED, "fsa_apply_host: call fsa_tensor_generate first");
  DeviceGuard dg;
  cudaError_t e = dg.set(p->device);
  const size_t vbytes = (size_t)p->n[0] * p->n[1] * p->n[2] * (p->dtype == FSA_F32 ? 4 : 8);
  // rho is staged in the Y region (free until the second pass writes it);
  // phi is produced there too (Y is dead once the fourth pass has read it).
  // DDI plans read rho again in their last pass: they stage it (and produce
  // phi, element by element in place) behind X and Y.
  void* X = p->ws;
  void* Y = (char*)p->ws + p->x_bytes;
  void* R = p->ddi >= 0 ? (void*)((char*)p->ws + align256(plan_workspace_bytes(p->n, p->dtype))) : Y;
  cudaStream_t s = (cudaStream_t)stream;
  if (e == cudaSuccess) e = cudaMemcpyAsync(R, rho_host, vbytes, cudaMemcpyHostToDevice, s);
  (void)X;
  (void)Y;
  if (e == cudaSuccess) e = plan_apply_graph(p, R, R, s);  // X = ws, Y = ws + x_bytes
  if (e == cudaSuccess) e = cudaMemcpyAsync(phi_host, R, vbytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_error(e, "fsa_apply_host");
  return FSA_OK;
}

}  // extern "C"
