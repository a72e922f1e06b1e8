// Internal declarations shared by the host-side translation units of libfsaconv.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/fsaconv.h"
#include "fsa_consts.h"

namespace fsa {

enum PassKind { kR2C = 0, kRowFwd = 1, kColMid = 2, kRowInv = 3, kC2R = 4, kNumPass = 5 };

// Tile geometry of one pass instance (lines per CTA, threads, shared bytes).
struct Geometry {
  int W = 0;
  int threads = 0;
  int smem = 0;
};

bool supported_n(int n);
int& autotune_mode();  // fsa_autotune_set: 0 defaults, 1 tune per plan, 2 / 3 force generation 1 / 2
// Kernel generation used for a pass of length M in a dtype: 1 = Stockham
// radix-8 (passes.cuh), 2 = two-step register kernels (passes2.cuh, FP32).
int kernel_variant(int pass, int M, fsa_dtype dt);
void set_kernel_variant(int pass, int M, fsa_dtype dt, int variant);
bool supported_M(int M);

// Per-precision launchers (passes_f32.cu / passes_f64.cu).  `M` is the
// transform length of the pass's axis; every job of a launch shares the grid.
// Each returns the launch error.
template <typename V> struct Passes {
  static cudaError_t prepare(int M);  // shared-memory opt-in and occupancy, current device
  static Geometry geometry(PassKind k, int M);
  static cudaError_t r2c_ax0(int M, const Jobs& jobs, long long C, cudaStream_t s);
  static cudaError_t row_fwd(int M, const Jobs& jobs, long long rows, cudaStream_t s);
  static cudaError_t col_mid(int M, const Jobs& jobs, int M2, int planes, cudaStream_t s);
  static cudaError_t row_inv(int M, const Jobs& jobs, long long rows, cudaStream_t s);
  static cudaError_t c2r_ax0(int M, const Jobs& jobs, long long C, cudaStream_t s);
  static cudaError_t init_twiddles();  // fills this TU's table on the current device
};

// The five apply passes for `count` solves sharing the grid n (plan.cu).
// With ev != nullptr (count <= kMaxJobs), six events are recorded: before the
// first pass and after each pass.
template <typename V>
cudaError_t group_passes(const int* n, int count, const void* const* rho, void* const* phi, void* const* X,
                         void* const* Y, const void* const* S, cudaStream_t s, cudaEvent_t* ev = nullptr);
cudaError_t plan_apply_passes(const fsa_plan* p, const void* rho, void* phi, cudaStream_t s);

// Drop cached batched graphs that refer to a plan (batched.cu).
void batched_forget_plan(const fsa_plan* p);

// Resident CTAs per SM for a kernel (cached per function), times the SM count.
int persistent_grid(const void* func, int threads, int smem, long long tiles);

// Tensor generation (tensor_gen.cu), all FP64.
cudaError_t tensorgen_prepare(int M);
cudaError_t tensorgen_init_twiddles();
cudaError_t tensorgen_run(const int n[3], const double L[3], double eps, double* oct64, void* out,
                          fsa_dtype dtype, cudaStream_t s);

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
  fsa_dtype dtype;
  int device;
  int generated;
  void* spectrum;
  size_t spectrum_bytes;
  void* ws;  // X then Y
  size_t ws_bytes;
  size_t x_bytes;
};
