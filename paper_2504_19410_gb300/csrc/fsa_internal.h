// Internal declarations shared by the host-side translation units of libfsaconv.
#pragma once
#include <vector>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/fsaconv.h"
#include "fsa_consts.h"

namespace fsa {

// Dimension of a kernel of Table 1 (2 for the plane kernels, else 3).
inline int kernel_dim(fsa_kernel k) {
  return (k == FSA_KERNEL_POISSON2D || k == FSA_KERNEL_COULOMB2D || k == FSA_KERNEL_BIHARMONIC2D ||
          k == FSA_KERNEL_YUKAWA2D)
             ? 2
             : 3;
}
inline bool kernel_has_param(fsa_kernel k) { return k == FSA_KERNEL_YUKAWA3D || k == FSA_KERNEL_YUKAWA2D; }

enum PassKind { kR2C = 0, kRowFwd = 1, kColMid = 2, kRowInv = 3, kC2R = 4, kNumPass = 5 };

// Tile geometry of one pass instance (lines per CTA, threads, shared bytes).
struct Geometry {
  int W = 0;
  int threads = 0;
  int smem = 0;
};

bool supported_n(int n);
int& autotune_mode();  // fsa_autotune_set: 0 defaults, 1 tune per plan, 2..5 force generation 1..4
// Kernel generation used for a pass of length M in a dtype: 1 = Stockham
// radix-8 (passes.cuh), 2 = two-step register kernels (passes2.cuh, FP32).
int kernel_variant(int pass, int M, fsa_dtype dt);
void set_kernel_variant(int pass, int M, fsa_dtype dt, int variant);
bool supported_M(int M);

// Launchers of one kernel instance (one arithmetic, one transform length M),
// registered at library load by the instance translation units (inst_*.cu)
// and looked up at launch.  Every job of a launch shares the grid.
struct Jobs;
struct PassFns {
  cudaError_t (*prepare)() = nullptr;  // shared-memory opt-in on the current device
  Geometry (*geometry)(PassKind) = nullptr;
  cudaError_t (*r2c)(const Jobs&, long long C, cudaStream_t) = nullptr;
  cudaError_t (*rowf)(const Jobs&, long long rows, cudaStream_t) = nullptr;
  cudaError_t (*colm)(const Jobs&, int M2, int planes, cudaStream_t) = nullptr;
  cudaError_t (*rowi)(const Jobs&, long long rows, cudaStream_t) = nullptr;
  cudaError_t (*c2r)(const Jobs&, long long C, cudaStream_t) = nullptr;
  // d = 2: middle pass and narrow-tile R2C / C2R (first generation only;
  // nullptr for the others)
  cudaError_t (*rowm)(const Jobs&, long long rows, cudaStream_t) = nullptr;
  cudaError_t (*r2c_plane)(const Jobs&, long long C, cudaStream_t) = nullptr;
  cudaError_t (*c2r_plane)(const Jobs&, long long C, cudaStream_t) = nullptr;
  // 3-D DDI (Sec. 5, Example 4): the kernel reading's middle pass and the
  // grid reading's C2R with the local term (every generation), and the grid
  // reading's unpadded passes of length M (first generation only)
  cudaError_t (*colm_ddi)(const Jobs&, int M2, int planes, cudaStream_t) = nullptr;
  // the middle pass for jobs that all share one spectrum (densities of one
  // plan): one spectrum read per column tile where the generation has it
  cudaError_t (*colm_shared)(const Jobs&, int M2, int planes, cudaStream_t) = nullptr;
  cudaError_t (*c2r_epi)(const Jobs&, long long C, cudaStream_t) = nullptr;
  cudaError_t (*r2c_per)(const Jobs&, long long C, cudaStream_t) = nullptr;
  cudaError_t (*rowf_per)(const Jobs&, long long rows, cudaStream_t) = nullptr;
  cudaError_t (*colm_per)(const Jobs&, int M2, int planes, cudaStream_t) = nullptr;
  cudaError_t (*rowi_per)(const Jobs&, long long rows, cudaStream_t) = nullptr;
  cudaError_t (*c2r_per)(const Jobs&, long long C, cudaStream_t) = nullptr;
  // fifth generation (FP32, transform length M on axes 0 and 2): the fused
  // outer pass pairs run by thread-block clusters (passes5.cuh), rho -> Y and
  // Y -> phi, in cluster configuration cfg < nfused (CTAs per cluster
  // fused_cs[cfg], threads per CTA fused_nt[cfg])
  cudaError_t (*fwd5)(int cfg, const Jobs&, int n1, cudaStream_t) = nullptr;
  cudaError_t (*inv5)(int cfg, const Jobs&, int n1, cudaStream_t) = nullptr;
  int nfused = 0;
  int fused_cs[4] = {0, 0, 0, 0};
  int fused_nt[4] = {0, 0, 0, 0};
};
// FP32 generations: 1 Stockham radix-8, 2 two-step register, 3 = 2 with the
// middle pass prefetching its next tile (cp.async), 4 = 3 with the row passes
// staging whole tiles by bulk asynchronous copies.
enum Arith {
  kArithF32G1 = 0,
  kArithF32G2 = 1,
  kArithF64 = 2,
  kArithDW = 3,
  kArithF32G3 = 4,
  kArithF32G4 = 5,
  kArithF32G5 = 6,  // the fused outer pass pairs only (fwd5 / inv5)
  kArithF32G6 = 7,  // generation 4 with the sixth-generation middle pass
  kArithF32G8 = 8,  // generation 4 with the eighth-generation (tensor-copy) middle pass
  kNumArith = 9
};
// The sixth-generation middle pass (passes6.cuh, inst_f32g6.cu) for
// transform length M, or null where it has no instance; k6_prepare sets its
// shared-memory opt-in on the current device.
using ColmFn = cudaError_t (*)(const Jobs&, int, int, cudaStream_t);
ColmFn k6_colm(int M);
cudaError_t k6_prepare(int M);
// The eighth-generation middle pass (passes8.cuh, inst_f32g8.cu): column tiles
// staged by one tiled bulk tensor copy each; null where it has no instance.
ColmFn k8_colm(int M);
ColmFn k8_colm_shared(int M);  // its form for densities of one plan (one spectrum read per tile)
using R2cFn = cudaError_t (*)(const Jobs&, long long, cudaStream_t);
R2cFn k8_r2c(int M);  // the R2C pass staged the same way
R2cFn k8_c2r(int M);  // and the C2R pass (same launcher signature)
cudaError_t k8_prepare(int M);
// The seventh generation (passes7.cuh, inst_f32g7.cu): row forward, middle
// and row inverse of FP32 grids with n1 = n2 as one kernel fed by a work
// dispenser.  k7_pipe_fn(M): its launcher for transform length M (null where
// it has no instance); jobs in = X, out = Y, S = spectrum, job 0's aux = the
// counter words (pipe_ctr_bytes at the end of job 0's workspace).
using PipeFn = cudaError_t (*)(const Jobs&, int n1, int K0, cudaStream_t);
PipeFn k7_pipe_fn(int M);
cudaError_t k7_prepare(int M);
// Bytes of a solve's workspace: X, Y, then (grids the seventh generation can
// run) its counter words for a launch of up to kMaxJobs solves.
size_t plan_workspace_bytes(const int* n, fsa_dtype dt);
size_t pipe_ctr_bytes(const int* n, fsa_dtype dt);
// Whether FP32 grids of transform length M run the seventh generation: 0 the
// separate passes, 1 the pipelined kernel (only when pinned by
// fsa_pipe_select; -1, unpinned, runs the separate passes).
int pipe_config(int M);
void set_pipe_config(int M, int c);
// W(k) by the radial integrals of Eq. Fourier-Symmetric with adaptive
// Gauss-Kronrod quadrature (radial_w.cpp).  radial_w_table: piecewise Chebyshev
// series of degree kWTableDegree on [0, kmax]; layout: the P + 1 panel edges,
// then P x (kWTableDegree + 1) coefficients (the first halved), P in *panels.
constexpr int kWTableDegree = 24;
long double u_minus_ueps(fsa_kernel kernel, long double lam, long double eps, long double r);
bool radial_w_value(fsa_kernel kernel, double lam, double eps, double k, double* w, double* err);
bool radial_w_table(fsa_kernel kernel, double lam, double eps, double kmax, std::vector<double>* table,
                    int* panels);
// The batched launcher's mixed-length path (mixed.cu, passes_mix.cuh): whether
// a plan can join it, and the five launches for `count` such solves.
bool mixed_eligible(const fsa_plan* p);
// pipelined: two halves of balanced work in six launches, else one launch per pass
cudaError_t mixed_passes(int count, const fsa_plan* const* plans, const void* const* rho, void* const* phi,
                         cudaStream_t s, bool pipelined);
int mixed_launches(int count, bool pipelined);  // launches mixed_passes makes for `count` solves
// fsa_batched_mode_set: 0 auto, 1 mixed one launch per pass, 2 shape groups, 3 mixed pipelined
int& batched_mode();
// The fused outer pass pair used for FP32 grids with n0 = n2 and transform
// length M = 2 n0 (dir 0 forward, 1 inverse): 0 = the separate passes, c >= 1
// = fused cluster configuration c - 1.  set_fused_config(M, dir, -1) leaves
// the choice to the tuner.
int fused_config(int M, int dir);
void set_fused_config(int M, int dir, int c);
// This device's fault word (Jobs::fault), allocated by prepare_device;
// ensure_device_fault_word allocates it if needed (current device).
unsigned int* device_fault_word();
unsigned int* ensure_device_fault_word();
void register_pass_fns(int arith, int M, PassFns f);
const PassFns& pass_fns(int arith, int M);  // prepare == nullptr if absent
void register_twiddle_init(cudaError_t (*init)());
cudaError_t init_all_twiddles();  // every instance unit's tables, current device

// Resident CTAs per SM for a kernel (cached per function), times the SM count.
int persistent_grid(const void* func, int threads, int smem, long long tiles);
// Grid policy of the calling host thread's launches: 0 = persistent grids
// (resident CTAs x SMs, the default), 1 = one CTA per tile, so that the
// blocks of a long solve retire one tile at a time and kernels of
// higher-priority streams get SMs between them (the serving loop's bulk lane).
int& launch_grid_mode();

// Per-launch trace for the profiler: an event before the first launch and
// after every launch, and the pass kind of each launch (intervals i -> i+1).
struct PassTrace {
  cudaEvent_t* ev = nullptr;
  signed char* kind = nullptr;
  int cap = 0;   // events available
  int used = 0;  // events recorded
};

// The five apply passes for `count` solves sharing the grid n (plan.cu).
template <typename V>
cudaError_t group_passes(const int* n, int count, const void* const* rho, void* const* phi, void* const* X,
                         void* const* Y, const void* const* S, cudaStream_t s, PassTrace* tr = nullptr,
                         long long chunk_bytes = 0);
cudaError_t plan_apply_passes(const fsa_plan* p, const void* rho, void* phi, cudaStream_t s);

// The five passes for `count` solves of one plan shape in the plan's
// arithmetic: FP32, native FP64, or double-word for FP64 plans with f64_dw.
// par[k]: solve k's DDI parameter block (3-D DDI plans; may be null otherwise).
cudaError_t run_group(const fsa_plan* shape, int count, const void* const* rho, void* const* phi,
                      void* const* X, void* const* Y, const void* const* S, cudaStream_t s,
                      PassTrace* tr = nullptr, const DdiPar* const* par = nullptr);
// The spectrum the apply kernels read (the double-word copy for f64_dw plans).
const void* plan_apply_spectrum(const fsa_plan* p);
// Converts an FP64 octant to double-word pairs (tensor_gen.cu).
cudaError_t spectrum_to_dw(const double* src, void* dst, size_t count, cudaStream_t s);

// Drop cached batched graphs that refer to a plan (batched.cu).
void batched_forget_plan(const fsa_plan* p);
// fsa_apply's graph cache (apply_graph.cu): the passes of a solve, replayed
// from a CUDA graph once its (plan, rho, phi) has been seen before;
// invalidate after a kernel selection changes; forget a destroyed plan.
cudaError_t plan_apply_graph(const fsa_plan* p, const void* rho, void* phi, cudaStream_t s);
void apply_graphs_invalidate();
int apply_graphs_generation();  // bumped by every invalidate
void apply_graphs_forget_plan(const fsa_plan* p);

// Tensor generation (tensor_gen.cu), all FP64.
cudaError_t tensorgen_prepare(int M);
// Look up (and so reserve) fsa_apply_noalloc's static scratch on device dev,
// which must be current; once per device (noalloc.cu).
cudaError_t noalloc_resolve(int dev);
cudaError_t tensorgen_init_twiddles();
// param: the kernel's parameter (the Yukawa lam), ignored by the others
cudaError_t tensorgen_run(fsa_kernel kernel, const int n[3], const double L[3], double eps, double param,
                          double* oct64, void* out, fsa_dtype dtype, cudaStream_t s,
                          const double* wtab = nullptr, int wtab_panels = 0);

// Twiddle table exp(-2 pi i k / 3072), k < 3072, computed on the host.
void host_twiddles(double* re, double* im);

// Thread-local error reporting.
fsa_status set_error(fsa_status st, const std::string& msg);
fsa_status cuda_error(cudaError_t e, const char* what);

}  // namespace fsa

struct fsa_plan {
  int n[3];
  double L[3];
  double h[3];
  double eps;
  double R0;
  double eps_bound;
  fsa_kernel kernel;
  double param;  // the kernel's parameter (the Yukawa lam), 0 if it has none
  int d;  // 3, or 2 for the plane kernels (then n[2] = 1 and the octant is (n0+1)(n1+1))
  fsa_dtype dtype;
  int device;
  int generated;
  void* spectrum;
  size_t spectrum_bytes;
  void* spectrum_dw;  // FP64 plans: the spectrum as double-word pairs
  int f64_dw;         // FP64 plans: 1 = double-word arithmetic, 0 = native FP64
  long long chunk_bytes;  // pass split: target bytes of one slab's X + Y (<= 0: no split)
  void* ws;  // X then Y (then, for DDI plans, the host path's staging of rho)
  size_t ws_bytes;
  size_t x_bytes;
  // fsa_apply_many: workspaces for densities 1 .. many_cap - 1 (X then Y each,
  // many_stride bytes apart); density 0 uses ws
  void* ws_many;
  int many_cap;
  size_t many_stride;
  // 3-D DDI (Sec. 5, Example 4): -1 = not a DDI plan, else the fsa_ddi_derivative
  int ddi;
  fsa::DdiPar* ddi_par;  // device: the DDI parameters (fsa_consts.h)
  double dipole_n[3], dipole_m[3];
  // fsa_plan_opts.w_quadrature: device copy of the W(k) table (radial_w.cpp)
  double* wtab;
  int wtab_panels;
};
