/*
 * libfsaconv -- GB300 (sm_103a) apply path of the far-field smooth
 * approximation (FSA) convolution solver of Liu & Zhang, "Fast convolution
 * solver based on far-field smooth approximation" (arXiv 2504.19410).
 *
 * The library computes the discrete aperiodic convolution of Sec. 2.3,
 * Eq. (DiscConv):
 *
 *     Phi_m = sum_{i in I_N} T_{m-i} rho_i ,   T = T^(1) + T^(2),
 *
 * on an n_0 x n_1 x n_2 grid x_{j,l} = h_j l, l = -n_j/2 .. n_j/2 - 1,
 * h_j = 2 L_j / n_j (Sec. 2, the uniform mesh; Sec. 2.4 for a box with
 * different L_j).  T^(1)_o = h_0 h_1 h_2 U^eps(|o.h|) (Sec. 2.1, Eq. Tensor1)
 * and T^(2) is the inverse DFT over the doubled grid of W(mu_p), the
 * whole-space Fourier transform of U - U^eps at mu_{p,j} = pi p_j / (2 L_j)
 * (Sec. 2.2, Eqs. Tensor2, FouTran; Table 1).  The kernel is the 3-D Coulomb
 * kernel U = 1/(4 pi r) with U^eps = U erf(r/eps) (Sec. 4, Eq. KerAppr).
 *
 * Arrays.  Densities rho and potentials phi are dense C-order arrays of
 * n_0 * n_1 * n_2 elements of the plan's dtype (axis 2 fastest), array index
 * i_j = l_j + n_j/2.  Every pointer named rho / phi below is a DEVICE pointer
 * unless the function name says _host.  The caller owns rho and phi.
 *
 * Sizes.  Each n_j must be even, 4 <= n_j <= 512, and of the form 2^a or
 * 3 * 2^a (the doubled length 2 n_j then factors into the radices 2, 3, 4
 * and 8 the FFT kernels implement).
 *
 * Errors.  Every call returns an fsa_status; no C++ exception crosses the
 * ABI.  On error a message is kept per thread (fsa_last_error).  Calls that
 * enqueue device work are asynchronous with respect to the host and return
 * FSA_ERR_CUDA if a launch fails; device faults surface on a later
 * synchronisation, as with any CUDA library.
 *
 * Streams.  fsa_stream_t is a cudaStream_t (NULL = the legacy default stream).
 */
#ifndef FSACONV_H
#define FSACONV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fsa_stream_t; /* same type as cudaStream_t */

typedef enum {
  FSA_OK = 0,
  FSA_ERR_INVALID_ARG = 1,    /* a size, pointer or option is out of range      */
  FSA_ERR_UNSUPPORTED = 2,    /* kernel x dimension not implemented             */
  FSA_ERR_EPS = 3,            /* eps fails the App. B far-field bound          */
  FSA_ERR_OOM = 4,            /* device allocation failed or over budget        */
  FSA_ERR_CUDA = 5,           /* a CUDA runtime call failed                     */
  FSA_ERR_NOT_GENERATED = 6,  /* fsa_apply before fsa_tensor_generate           */
  FSA_ERR_BUSY = 7,           /* serving queue full                             */
  FSA_ERR_TIMEOUT = 8,        /* a host-side wait ran out                       */
  FSA_ERR_DEVICE_TIMEOUT = 9, /* a bounded device-side wait gave up             */
  FSA_ERR_NOT_FOUND = 10      /* unknown serving ticket                         */
} fsa_status;

typedef enum {
  FSA_KERNEL_COULOMB3D = 0,    /* d = 3: U = 1/(4 pi r), U^eps = U erf(r/eps) (Table 1)      */
  FSA_KERNEL_BIHARMONIC3D = 1, /* d = 3: U = r/(8 pi), U^eps = U erf(r/eps) (Table 1; Ex. 4) */
  FSA_KERNEL_POISSON2D = 2,    /* d = 2: U = -ln(r)/(2 pi),                                  */
                               /* U^eps = -(ln r + E1(r^2/eps^2)/2)/(2 pi) (Eq. lnrAppr)      */
  FSA_KERNEL_COULOMB2D = 3,    /* d = 2: U = 1/(2 pi r), U^eps = U erf(r/eps) (Table 1)       */
  FSA_KERNEL_BIHARMONIC2D = 4, /* d = 2: U = -r^2 (ln r - 1)/(8 pi),                          */
                               /* U^eps = -r^2 (ln r + E1(r^2/eps^2)/2 - 1)/(8 pi) (Table 1)  */
  FSA_KERNEL_DDI3D = 5,        /* d = 3: the dipole-dipole kernel of Sec. 5, Example 4,       */
                               /* through the Coulomb kernel; see fsa_plan_create_ddi3d      */
  FSA_KERNEL_YUKAWA3D = 6,     /* d = 3: U = exp(-lam r)/(4 pi r) (Example 4)                 */
  FSA_KERNEL_YUKAWA2D = 7      /* d = 2: U = K0(lam r)/(2 pi) (Example 4).  For both:         */
                               /* U^eps = U convolved with the Gaussian of transform          */
                               /* exp(-k^2 eps^2/4) (the heat-kernel integral of U from       */
                               /* t = eps^2/4), W = (1 - exp(-(k^2+lam^2) eps^2/4))/(k^2+lam^2); */
                               /* lam = fsa_plan_opts.kernel_param.  The paper states neither   */
                               /* lam nor its window for these kernels (Sec. 4, Eq. GeneralApprox1) */
} fsa_kernel;

/* How a 3-D DDI plan discretises d_n d_m rho (Sec. 5, Example 4, which
 * computes the DDI potential as Phi = -(m.n) rho - 3 (1/(4 pi |x|)) * (d_n d_m rho),
 * d_n = n . grad, and does not say how d_n d_m rho is formed). */
typedef enum {
  FSA_DDI_GRID = 0,  /* spectral d_n d_m rho on the n-point grid (period 2 L_j,             */
                     /* multiplier -(k.n)(k.m), k_j = pi q_j / L_j, Nyquist q_j = -n_j/2,  */
                     /* real part), then the Coulomb solve: reproduces Table 5's 3-D row.  */
                     /* Ten passes: five of length n_j, five of the Coulomb solve         */
  FSA_DDI_KERNEL = 1 /* the same derivative taken of the Coulomb convolution on the       */
                     /* doubled grid (period 4 L_j, k_j = pi q_j / (2 L_j)): the multiplier */
                     /* -3 S(k) (-(k.n)(k.m)) - (m.n) / (8 n0 n1 n2) in the middle pass,   */
                     /* the five passes of a Coulomb solve.  Same accuracy as FSA_DDI_GRID */
                     /* (round-off at h = 1/4 in Table 5's case), different coarse-grid   */
                     /* aliasing                                                           */
} fsa_ddi_derivative;

typedef enum {
  FSA_F32 = 0, /* rho, phi, stored spectrum and FFT arithmetic in FP32 */
  FSA_F64 = 1  /* the same in FP64                                      */
} fsa_dtype;

typedef struct {
  double eps;     /* FSA parameter; 0 selects min(1, R0/6), R0 = min_j 2 L_j     */
  double eps_tol; /* App. B bound R0^2 f(R0/eps) must not exceed this;         */
                  /* 0 selects App. B's 1e-16 for FSA_F64 plans and 1e-8 for  */
                  /* FSA_F32 plans; a negative value disables the check        */
  int device;     /* CUDA device ordinal; -1 = the calling thread's current one */
  double kernel_param; /* the Yukawa kernels' lam (> 0; 0 selects 1); ignored by  */
                       /* the other kernels                                         */
  int l2_chunk_mb; /* pass split: run the three middle passes per slab of planes   */
                   /* whose intermediates take about this many MB, so they stay  */
                   /* in L2; 0 or negative = one slab (the default: slabs of     */
                   /* 8-64 MB measured 1.3-3.6x slower at 256^3 on GB300, the    */
                   /* small slab launches cannot fill the GPU)                   */
  int w_quadrature; /* 0 (default): W from its closed form (Table 1; Ex. 4);     */
                    /* 1: W by the radial integral of Eq. Fourier-Symmetric with  */
                    /* adaptive Gauss-Kronrod quadrature on the host, tabulated   */
                    /* as piecewise Chebyshev series of k and evaluated on the    */
                    /* device (the paper's route for kernels without a closed     */
                    /* form; see fsa_radial_w)                                    */
} fsa_plan_opts;

typedef struct fsa_plan fsa_plan;

typedef struct {
  int n[3];                 /* grid points per axis                                   */
  double L[3];              /* box half-widths                                        */
  double h[3];              /* mesh steps 2 L_j / n_j                                 */
  double eps;               /* the FSA parameter in use                               */
  double R0;                /* min_j 2 L_j (Sec. 1)                                   */
  double eps_bound;         /* App. B: R0^2 f(R0/eps)                                 */
  fsa_dtype dtype;
  int device;
  int generated;            /* 1 once fsa_tensor_generate has been enqueued           */
  int arithmetic;           /* 0 FP32; FP64 plans: 1 native FP64, 2 double-word       */
  int launches_per_apply;   /* kernel launches of one fsa_apply: 2 + 3 x plane slabs, */
                            /* one fewer per fused outer pair (fused_fwd, fused_inv), */
                            /* 3 with the pipelined middle passes (pipe)              */
  size_t workspace_bytes;   /* device scratch the plan owns                           */
  size_t spectrum_bytes;    /* device bytes of the stored spectrum octant             */
  const void* spectrum;     /* device pointer: (n0+1) x (n1+1) x (n2+1) dtype, C order */
  fsa_kernel kernel;        /* the plan's kernel                                      */
  int d;                    /* 3, or 2 for the plane kernels (then n[2] = 1, the      */
                            /* spectrum octant is (n0+1) x (n1+1), 3 launches/apply)  */
  double kernel_param;      /* the Yukawa lam in use; 0 for the other kernels         */
  int many_capacity;        /* densities one fsa_apply_many call may take (1 + the    */
                            /* workspaces added by fsa_plan_reserve)                  */
  int ddi_derivative;       /* FSA_KERNEL_DDI3D plans: their fsa_ddi_derivative; -1   */
  double dipole_n[3];       /* FSA_KERNEL_DDI3D plans: n and m; zero otherwise        */
  double dipole_m[3];
  int fused_fwd;            /* the outer forward pair in use (fsa_fused_select): 0    */
  int fused_inv;            /* separate passes, c >= 1 fused configuration c - 1     */
  int w_quadrature;         /* 1 if W comes from the quadrature table, else 0         */
  int w_panels;             /* that table's Chebyshev panels (0 without it)           */
  int pipe;                 /* 1 if the middle passes run as the pipelined kernel    */
                            /* (fsa_pipe_select), else 0                              */
} fsa_plan_info;

/* Create a plan (the "Precomp" object of Sec. 5, Example 2) for the grid
 * n[0..d-1] on the box prod_j [-L_j, L_j].  d is the kernel's dimension: 3
 * for the 3-D kernels, 2 for the plane kernels (Poisson, Coulomb, biharmonic
 * of Table 1), whose solves run R2C along axis 0, one middle pass along
 * axis 1 (forward, multiply, inverse) and C2R (Sec. 2.3 with d = 2).  The plan owns,
 * on the chosen device, the spectrum octant and the apply workspace
 * (fsa_plan_info.workspace_bytes); both are freed by fsa_plan_destroy.
 * kernel: one of Table 1's kernels (FSA_KERNEL_DDI3D plans come from
 * fsa_plan_create_ddi3d); the apply path is the same for all kernels of one
 * dimension, only the generated spectrum differs.
 * eps follows Remark 2.1 / App. B: the plan computes the far-field integral
 * int_{R0}^inf |U - U^eps| r^2 dr (fsa_appendix_b_bound_kernel) and rejects
 * eps with FSA_ERR_EPS when it exceeds opts->eps_tol.  opts may be NULL.
 * Errors: FSA_ERR_INVALID_ARG (out == NULL, d != 3, unsupported n_j,
 * L_j <= 0, eps < 0), FSA_ERR_UNSUPPORTED (kernel), FSA_ERR_EPS,
 * FSA_ERR_OOM, FSA_ERR_CUDA.  On error *out is set to NULL. */
fsa_status fsa_plan_create(fsa_plan** out, fsa_kernel kernel, int d, const double* L,
                           const int* n, fsa_dtype dtype, const fsa_plan_opts* opts);

/* A plan for the 3-D dipole-dipole potential of Sec. 5, Example 4:
 *   Phi = -(m.n) rho - 3 (1/(4 pi |x|)) * (d_n d_m rho),
 * the kernel U(x) = (3/(4 pi)) (m.n - 3 (x.m)(x.n)/|x|^2) / |x|^3 applied through
 * the 3-D Coulomb kernel's FSA tensor (same spectrum, eps rule and App. B
 * check as FSA_KERNEL_COULOMB3D).  dipole_n, dipole_m: 3 doubles each (host),
 * finite (the paper takes unit vectors; any vectors are accepted, the
 * potential is bilinear in them).  derivative: see fsa_ddi_derivative; the
 * grid reading needs n_j >= 8.  fsa_tensor_generate, fsa_apply,
 * fsa_apply_host, fsa_apply_noalloc and fsa_apply_batched then compute the
 * DDI potential; the plan's workspace holds n0 n1 n2 more dtype elements
 * (fsa_apply_host stages rho there).  Serving requests do not take DDI
 * plans.  Errors as fsa_plan_create; FSA_ERR_INVALID_ARG also for NULL or
 * non-finite dipoles, an unknown derivative, or n_j < 8 with FSA_DDI_GRID. */
fsa_status fsa_plan_create_ddi3d(fsa_plan** out, const double* L, const int* n, fsa_dtype dtype,
                                 const double* dipole_n, const double* dipole_m,
                                 fsa_ddi_derivative derivative, const fsa_plan_opts* opts);

/* Generate the kernel tensor's spectrum on the device, in FP64, and store it
 * in the plan's dtype (Sec. 2.1-2.3: T^(1) by the trapezoid rule, T^(2) from
 * W; the spectrum of T is DFT(T^(1)) + W because T^(2) = iDFT(W)).  Stored:
 * S[p] = (DFT_{2n}(T^(1))[p] + W(|mu_p|)) / (8 n0 n1 n2) for p_j in [0, n_j];
 * T is real and even per axis (Sec. 2.3), so this octant is the whole
 * spectrum.  The DFT of the even tensor is a separable DCT-I, computed with
 * the library's FFT kernels.  Asynchronous on stream; idempotent. */
fsa_status fsa_tensor_generate(fsa_plan* plan, fsa_stream_t stream);

/* Phi = T * rho (Eq. DiscConv) by zero-padding to 2n per axis, FFT, multiply
 * by the stored spectrum and inverse FFT, keeping the first n_j outputs per
 * axis (Sec. 2.3).  rho, phi: device arrays of n0*n1*n2 plan-dtype elements;
 * phi == rho is allowed.  Uses the plan's workspace, so calls on one plan
 * must not overlap on the GPU.  Asynchronous on stream.  From the second
 * call with the same (plan, rho, phi) on, the passes are replayed from a
 * CUDA graph captured at that call (fsa_apply_graphs_set).
 * Errors: FSA_ERR_INVALID_ARG (NULL pointer), FSA_ERR_NOT_GENERATED,
 * FSA_ERR_CUDA. */
fsa_status fsa_apply(const fsa_plan* plan, const void* rho, void* phi, fsa_stream_t stream);

/* Graph replay of repeated solves (no counterpart in the paper: it concerns
 * the launches, not the method).  With enable = 1 (the default), fsa_apply
 * and fsa_apply_host capture the pass launches of a (plan, rho, phi) triple
 * into a CUDA graph on the second call with that triple and replay the graph
 * on later calls (one graph launch instead of one launch per pass; results
 * bit-equal to direct launches).  A graph keeps the kernels selected when it
 * was captured; fsa_autotune_set, fsa_fused_select and fsa_pipe_select make
 * later calls capture anew.  Up to 64 graphs per device are kept (least
 * recently used dropped); a plan's graphs are dropped by fsa_plan_destroy.
 * enable = 0: every call launches its passes directly.
 * FSA_ERR_INVALID_ARG for enable other than 0 or 1. */
fsa_status fsa_apply_graphs_set(int enable);

/* fsa_apply for callers that cannot have device memory allocated for them
 * (the paper has no counterpart: this is a deployment variant).  Same result
 * as fsa_apply on the same plan, but the two intermediate arrays live in a
 * 16 MiB static __device__ array of the library instead of the plan's
 * workspace, and the call allocates nothing.  Size limit: the workspace
 * 6 (n0+1) n1 n2 s bytes (s = 4 for FP32, 8 for FP64) must fit in 16 MiB,
 * e.g. grids up to 64^3 in both precisions; larger grids get
 * FSA_ERR_INVALID_ARG.  The array is reserved on a device (its address
 * looked up with cudaGetSymbolAddress, which loads its module) when the
 * first plan is created there, so create plans before the caller's
 * allocator takes the remaining memory; if that lookup failed, the first
 * call here retries it, and that call should come before any stream
 * capture.  All calls on a device share the array and it keeps the
 * last call's contents; nothing in it needs to start at zero, but calls that
 * overlap on the GPU race, so order them (one stream, or events).
 * Errors as fsa_apply. */
fsa_status fsa_apply_noalloc(const fsa_plan* plan, const void* rho, void* phi, fsa_stream_t stream);

/* fsa_apply with HOST buffers: copies rho_host to the device, applies, copies
 * the result to phi_host, all enqueued on stream (pinned host memory gives
 * asynchronous copies).  The caller must synchronise the stream before
 * reading phi_host.  Staging goes through the plan's workspace. */
fsa_status fsa_apply_host(const fsa_plan* plan, const void* rho_host, void* phi_host,
                          fsa_stream_t stream);

/* Apply count plans to count densities in one launch sequence.  Plans may
 * differ in n, L, eps and dtype but must share a device.  The requests whose
 * plan is an FP32 plan of d = 3 (not DDI, no pass split) with every transform
 * length 2 n_j in {128, 192, 256, 384, 512} can share one persistent launch
 * per pass over the concatenated tile lists of all of them, whatever their
 * sizes (the mixed path; whether a batch takes it is fsa_batched_mode_set's
 * choice, by default timed on the batch's first call); such a request's
 * result matches
 * fsa_apply(plans[k], rho[k], phi[k]) within FP32 round-off (the same
 * transforms, factored as 16 x (M / 16)), not bit for bit.  The other
 * requests are grouped by grid and dtype, each group's passes run as
 * grid-strided persistent kernels over the tiles of all its requests, on
 * concurrent streams, and each of their results equals fsa_apply's bit for
 * bit.  Either sequence is captured once per batch signature (plans and
 * buffers) into a CUDA graph and replayed; after fsa_autotune_set,
 * fsa_fused_select or fsa_pipe_select the next call captures the batch again
 * with the newly selected kernels.  Uses each plan's workspace, so a plan may
 * appear at most once per call (FSA_ERR_INVALID_ARG otherwise). */
fsa_status fsa_apply_batched(const fsa_plan* const* plans, const void* const* rho,
                             void* const* phi, int count, fsa_stream_t stream);

/* How fsa_apply_batched schedules the requests that fit the mixed-length
 * kernels (no counterpart in the paper: the batched path's schedule choice;
 * process-wide, applies to batch signatures captured afterwards).
 * mode 0 (default, auto): the first call of a batch signature captures the
 * candidates of modes 1 and 2, launches each twice (the second timed) and
 * keeps the faster; that call's results are from the kept schedule.
 * mode 1: the mixed-length requests in one launch per pass, five in all.
 * mode 2: no mixed path; every request in its shape group (one persistent
 * launch per pass per group, groups on concurrent streams).
 * mode 3: the mixed-length requests software-pipelined in two halves of
 * balanced work, six launches, the middle four each running one half's pass
 * beside the other's previous pass with their tiles interleaved.
 * Results of modes 1 and 3 are the same bits; mode 2 gives fsa_apply's bits.
 * Errors: FSA_ERR_INVALID_ARG (other modes). */
fsa_status fsa_batched_mode_set(int mode);

/* How many kernel launches fsa_apply_batched makes for these plans (no
 * counterpart in the paper: launch accounting for the batched path): five per
 * 64 requests of the mixed path, plus each group's launches per apply per 64
 * requests (six for a pipelined batch), under the schedule
 * fsa_batched_mode_set selects (mode 0: the one kept for these plans once a
 * batch of them has run, the mixed path before).  Host only.  Errors:
 * FSA_ERR_INVALID_ARG (NULL). */
fsa_status fsa_apply_batched_launches(const fsa_plan* const* plans, int count, int* launches);

/* Many densities through one plan (the paper's Execution phase repeated with one
 * cached tensor, e.g. the steps of a time-dependent solver).  fsa_plan_reserve
 * allocates device workspace so that fsa_apply_many can take up to `count`
 * densities at once (count - 1 more copies of the plan's X and Y regions;
 * fsa_plan_info.workspace_bytes does not include them); it never shrinks and
 * may be called again to grow.  fsa_apply_many(plan, rho, phi, count) computes
 * phi[k] = T * rho[k] (the plan's kernel, DDI plans included) for k < count in
 * one launch sequence: every pass is one persistent launch over the tiles of
 * all densities, and the middle pass takes a column tile for every density in
 * turn, reading the tile's spectrum values once (FP32, generations 3 and 4).
 * Results equal fsa_apply's bit for bit.  rho[k], phi[k]: device arrays as for
 * fsa_apply, 16-byte aligned; phi[k] == rho[k] is allowed, other overlaps are
 * not.  Asynchronous on stream; calls on one plan must not overlap on the GPU.
 * Errors: FSA_ERR_INVALID_ARG (count < 1 or above the capacity, NULL or
 * misaligned pointers), FSA_ERR_NOT_GENERATED, FSA_ERR_OOM (reserve),
 * FSA_ERR_CUDA. */
fsa_status fsa_plan_reserve(fsa_plan* plan, int count);
fsa_status fsa_apply_many(const fsa_plan* plan, const void* const* rho, void* const* phi, int count,
                          fsa_stream_t stream);

fsa_status fsa_plan_info_get(const fsa_plan* plan, fsa_plan_info* info);
fsa_status fsa_plan_destroy(fsa_plan* plan); /* NULL is a no-op */

/* Copy the stored spectrum octant ((n0+1)(n1+1)(n2+1) plan-dtype values,
 * C order, p_j in [0, n_j]) to dst, a device or host buffer of at least
 * fsa_plan_info.spectrum_bytes bytes (cudaMemcpyDefault).  Asynchronous on
 * stream for device or pinned destinations.  FSA_ERR_INVALID_ARG if
 * nbytes is too small. */
fsa_status fsa_plan_spectrum_copy(const fsa_plan* plan, void* dst, size_t nbytes, fsa_stream_t stream);

/* App. B far-field bound for the 3-D Coulomb kernel: R0^2 f(R0/eps) with
 * f(c) = (1/(4 pi c^2)) int_c^inf s erfc(s) ds (host-only; NaN for
 * non-positive arguments).  fsa_plan_create checks it against eps_tol. */
double fsa_appendix_b_bound(double R0, double eps);

/* The same far-field integral int_{R0}^inf |U - U^eps| r^2 dr for a kernel of
 * Table 1: Coulomb as above; 3-D biharmonic (App. B works out only Coulomb;
 * the same integral of r erfc(r/eps)/(8 pi)) =
 * (eps^4 / (8 pi)) int_c^inf s^3 erfc(s) ds, c = R0/eps, in closed form
 * erfc(c) (3/16 - c^4/4) + exp(-c^2) (c^3/2 + 3c/4) / (2 sqrt(pi)).
 * Host-only; NaN for non-positive arguments or an unknown kernel. */
double fsa_appendix_b_bound_kernel(fsa_kernel kernel, double R0, double eps);

/* The same for a kernel with a parameter (the Yukawa kernels: param = lam):
 * int_{R0}^inf (U - U^eps) r^{d-1} dr with U - U^eps the heat-kernel integral
 * below t = eps^2/4, by Gauss-Legendre quadrature after swapping the order:
 * d = 3: int_0^{eps^2/4} exp(-lam^2 t) (4 pi t)^{-3/2} (2 t R0 exp(-R0^2/(4t))
 *        + 2 sqrt(pi) t^{3/2} erfc(R0/(2 sqrt t))) dt;
 * d = 2: (1/(2 pi)) int_0^{eps^2/4} exp(-lam^2 t - R0^2/(4t)) dt.
 * Other kernels: as fsa_appendix_b_bound_kernel.  NaN for non-positive
 * arguments. */
double fsa_appendix_b_bound_kernel_param(fsa_kernel kernel, double param, double R0, double eps);

const char* fsa_status_string(fsa_status s);
const char* fsa_last_error(void); /* calling thread's last error message ("" if none) */

/* ------------------------------------------------------------ profiling -- */
/* Per-pass timing with CUDA events on the launching stream.  A profiler holds
 * 512 events per step for up to max_steps (1..4096) steps (cudaEventCreate:
 * no device memory).  fsa_apply_profiled is fsa_apply plus an event before
 * the first launch and after every launch, each tagged with its pass;
 * fsa_profiler_read synchronises and returns, averaged over the recorded
 * steps, the time of each pass (pass_ms[5]: r2c_ax0, row_fwd, col_mid,
 * row_inv, c2r_ax0; a pass run in several plane slabs is the sum of its
 * launches) and of the whole step (step_ms), then resets.  FSA_ERR_BUSY if
 * more than max_steps steps are recorded before a read. */
typedef struct fsa_profiler fsa_profiler;
fsa_status fsa_profiler_create(fsa_profiler** out, int max_steps);
fsa_status fsa_apply_profiled(const fsa_plan* plan, const void* rho, void* phi, fsa_stream_t stream,
                              fsa_profiler* prof);
fsa_status fsa_profiler_read(fsa_profiler* prof, double* pass_ms, double* step_ms, int* steps);
fsa_status fsa_profiler_destroy(fsa_profiler* prof);

/* Kernel selection.  FP32 passes exist in four generations: 1 = Stockham
 * radix-8 (three shared-memory stages per transform), 2 = two register-resident
 * steps M = R1 x R2 (one exchange per transform), 3 = generation 2 with the
 * middle pass prefetching its next tile asynchronously, 4 = generation 3 with
 * the row passes staging whole tiles by double-buffered bulk asynchronous
 * copies; generation 6 = generation 4 with a middle pass that splits the
 * padded and cropped step of generation 2 into two half tasks per line, so
 * each thread holds half the values and twice the warps fit on an SM
 * (lengths 128, 192, 256, 384, 512; generation 4's middle pass elsewhere);
 * generation 8 = generation 4 with a middle pass and the axis-0 R2C and C2R
 * passes whose column tiles are staged by tiled bulk tensor copies (TMA),
 * bit-equal to generation 2's (same lengths; one tensor map per solve of a
 * launch).
 * mode 1 (default): each new FP32 plan times every generation for
 * each of its passes on its own workspace at creation and keeps the fastest
 * per (pass, length); choices persist for the process.  mode 0: untuned
 * passes use generation 2.  mode 2 / 3 / 4 / 5 / 6 / 7: force generation
 * 1 / 2 / 3 / 4 / 6 / 8 for every FP32 pass.  FP64 plans compute either in native FP64 or in
 * double-word arithmetic (two floats, 48-bit significand, on the FP32 pipes;
 * see fsa_plan_info.arithmetic): one choice per grid shape per process, timed
 * on the first plan of the shape in mode 1, double-word in mode 0, native in
 * mode 2, double-word in modes 3 to 7.  FSA_ERR_INVALID_ARG for other modes.
 * Not thread-safe against concurrent launches. */
fsa_status fsa_autotune_set(int mode);

/* Fused outer passes (FP32 plans of d = 3 with n0 = n2 and transform length
 * M = 2 n0 in {64, 128, 256, 384, 512}).  The five passes of Sec. 2.3 stay the same
 * transforms in the same order, but the pad + R2C along axis 0 and the
 * forward axis-2 transform run as one kernel, and so do the inverse axis-2
 * transform and the C2R along axis 0 + crop: a thread-block cluster holds one
 * i1-slab of the half spectrum X in the distributed shared memory of its CTAs,
 * so X never goes to HBM.
 * fsa_fused_configs returns how many cluster configurations exist for length
 * M (0: none) and writes, for the first min(count, cap) of them, the CTAs per
 * cluster and the threads per CTA (either pointer may be NULL).
 * fsa_fused_select(M, dir, c) pins the pair used for direction dir (0 forward,
 * 1 inverse, 2 both): c = 0 the separate passes, c >= 1 configuration c - 1,
 * c = -1 unpinned (the default).  Unpinned, autotune mode 1 times the separate
 * passes and every configuration on the first plan of the length and keeps the
 * fastest; mode 0 runs the separate passes; modes 2 to 5 always run the
 * separate passes of the forced generation, pinned or not.  The pass profiler reports a
 * fused pair under row_fwd / row_inv (r2c_ax0 / c2r_ax0 then read 0).
 * Plans with a pass split (l2_chunk_mb), DDI, FP64 and d = 2 plans use the
 * separate passes.  FSA_ERR_INVALID_ARG for a length without configurations,
 * dir outside 0..2 or c outside -1..count.  Not thread-safe against
 * concurrent launches. */
int fsa_fused_configs(int M, int* cluster_ctas, int* threads, int cap);
fsa_status fsa_fused_select(int M, int dir, int c);

/* Pipelined middle passes (FP32 plans of d = 3 with n1 = n2 and transform
 * length M = 2 n2 in {128, 192, 256, 384, 512}).  The forward axis-2
 * transform, the axis-1 middle pass with the spectrum multiply and the
 * inverse axis-2 transform of Sec. 2.3 stay the same transforms with the same
 * arithmetic (results bit-equal to the separate passes'), but run as one
 * persistent kernel whose CTAs take tiles of one axis-0 frequency plane at a
 * time from a work counter, each tile after the tiles of its plane it
 * depends on: the planes in flight stay in L2, and the row tiles share the
 * SMs with the middle tiles.  fsa_pipe_select(M, c): c = 1 the pipelined
 * kernel, 0 or -1 (the default) the separate passes; autotune modes 2 to 6
 * always run the separate passes of the forced generation.  (Measured on a
 * GB300 at 256^3: the pipelined kernel moves 0.55 GB through HBM instead of
 * 1.27 GB but takes 0.42 ms against 0.37 ms for the three passes, which are
 * bound by instruction issue and latency, not by HBM; it is not timed by the
 * tuner.)  A fused outer pair (fsa_fused_select) in use takes precedence.  The pass profiler reports the pipelined kernel under col_mid
 * (row_fwd / row_inv then read 0).  FSA_ERR_INVALID_ARG for a length without
 * the kernel or c outside -1..1.  Not thread-safe against concurrent
 * launches. */
fsa_status fsa_pipe_select(int M, int c);

/* Device-side wait status (no counterpart in the paper: it reports on the
 * kernels, not on the method).  Kernels that wait on an mbarrier for their own
 * asynchronous copies bound every wait (about 1 s); a CTA whose wait gives up
 * records FSA_ERR_DEVICE_TIMEOUT's cause in a per-device word and returns
 * instead of hanging, leaving its part of that solve's output undefined.
 * *code receives the word (0 = no wait gave up; bit 0 = an mbarrier wait
 * timed out) for `device` (-1 = current); clear != 0 resets it.  Read after
 * the work of interest has completed (e.g. after synchronizing its stream):
 * the read does not wait for other streams.  Errors: FSA_ERR_INVALID_ARG
 * (code NULL), FSA_ERR_CUDA. */
fsa_status fsa_device_fault(int device, unsigned int* code, int clear);

/* Self-test of the bounded device-side wait (no counterpart in the paper: it
 * checks the library's own safeguard).  On `device` (-1 = current) one CTA
 * waits, with a bound of about 1 ms, on an mbarrier that nothing completes,
 * takes the give-up path of the bulk-copy row passes (records the timeout in
 * the device's fault word, returns) and the host reads the word: *code = 1
 * (bit 0, an mbarrier wait timed out) when the safeguard works.  The word is
 * cleared again before return.  Synchronous; nothing faults or hangs.
 * Errors: FSA_ERR_INVALID_ARG (code NULL), FSA_ERR_CUDA. */
fsa_status fsa_wait_selftest(int device, unsigned int* code);

/* W(k) of `kernel` (Table 1's kernels, the Yukawa kernels with lam =
 * kernel_param, 0 selecting 1; a DDI kernel as Coulomb) by the radial Fourier
 * integral of U - U^eps (Sec. 2.2, Eq. Fourier-Symmetric: 4 pi int (U - U^eps)
 * sin(kr)/(kr) r^2 dr in 3-D, 2 pi int (U - U^eps) J0(kr) r dr in 2-D), on
 * the host in long double, by adaptive 15-point Gauss-Kronrod quadrature
 * (see fsa_gauss_kronrod15) over [0, 7 eps].  *err_estimate (may be NULL):
 * the summed |Kronrod - Gauss| of the final panels at this k.  This is the
 * routine behind fsa_plan_opts.w_quadrature.  Errors: FSA_ERR_INVALID_ARG. */
fsa_status fsa_radial_w(fsa_kernel kernel, double kernel_param, double eps, double k, double* w,
                        double* err_estimate);

/* The 15-point Gauss-Kronrod rule on [-1, 1] the radial quadrature uses,
 * computed (not tabulated): the Kronrod extension of the 7-point Gauss-Legendre
 * rule, new nodes from the Stieltjes polynomial, weights from exactness on the
 * Legendre polynomials of degree < 15.  nodes ascending; gauss_weights is 0 at
 * the 8 Kronrod-only nodes.  Each array holds 15 doubles.  Errors:
 * FSA_ERR_INVALID_ARG (NULL). */
fsa_status fsa_gauss_kronrod15(double* nodes, double* kronrod_weights, double* gauss_weights);

/* Measured ALU peak (no counterpart in the paper: the denominator of the
 * ALU rooflines of the FP64 tier, whose double-word passes run on the FP32
 * pipes and whose native passes run on the FP64 pipe).  kind 0: FP32 fused
 * multiply-add, kind 1: FP64 fused multiply-add, kind 2: the paired FP32
 * fused multiply-add (fma.rn.f32x2, two FMAs per instruction; counted as 2).  On `device` (-1 = current)
 * every resident thread runs 8 independent FMA chains for a fixed count;
 * the best of 3 timed launches (after one warm-up) gives *lane_ops_per_s
 * (one FMA = one lane operation = 2 flops); *ms (may be NULL) receives that
 * launch's time.  Synchronous, a few ms per kind.  Errors:
 * FSA_ERR_INVALID_ARG (NULL result, kind not 0, 1 or 2), FSA_ERR_CUDA. */
fsa_status fsa_measure_alu_peak(int device, int kind, double* lane_ops_per_s, float* ms);

/* ---------------------------------------------------------------- serving -- */

typedef struct fsa_server fsa_server;

typedef struct {
  int max_inflight;        /* requests on the GPU at once (0 = 64)                    */
  int streams;             /* device streams the requests are spread over (0 = 8)    */
  double hbm_fraction;     /* admit while plans + workspaces fit this share of the
                              device memory free now plus what the server holds,
                              re-read before each admission round (0 = 0.9)      */
  size_t hbm_budget_bytes; /* hard cap on server-held device bytes (0 = none)        */
  int plan_cache_max;      /* plans kept resident (0 = 64), least recently used out  */
  int queue_max;           /* pending requests before FSA_ERR_BUSY (0 = 1 << 20)     */
  int device;              /* -1 = current                                           */
  int policy;              /* 0 = size-aware lanes (default), 1 = round robin: see    */
                           /* fsa_serve_create                                        */
} fsa_serve_opts;

typedef struct {
  fsa_kernel kernel; /* any kernel but FSA_KERNEL_DDI3D (its plans need dipoles) */
  int d;          /* the kernel's dimension: 3, or 2 for the plane kernels (n[2], L[2] ignored) */
  double L[3];
  int n[3];
  fsa_dtype dtype;
  double eps;     /* 0 = default rule */
  const void* rho; /* device, caller-owned until the ticket is DONE or FAILED */
  void* phi;       /* device, caller-owned */
  double kernel_param; /* Yukawa kernels: lam (0 selects 1); ignored by the others */
} fsa_request;

typedef enum {
  FSA_REQ_QUEUED = 0,
  FSA_REQ_RUNNING = 1,
  FSA_REQ_DONE = 2,
  FSA_REQ_FAILED = 3
} fsa_req_state;

typedef struct {
  double submit_s; /* host clock (s, monotonic) at submit   */
  double admit_s;  /* when its work was enqueued            */
  double done_s;   /* when its completion event was seen    */
  int plan_hit;    /* 1 if its plan was already resident    */
  fsa_status status;
} fsa_req_times;

typedef struct {
  uint64_t submitted, completed, failed, plan_hits, plan_misses;
  size_t device_bytes_held; /* plans + workspaces */
  int inflight;
  int queued;
} fsa_serve_stats;

/* A serving loop: one host thread admits queued requests while their plan
 * (on a cache miss: the spectrum octant, for FP64 plans also its double-word
 * copy, and the generation scratch) and workspace fit the HBM budget and
 * fewer than max_inflight are on the GPU, launches each on one of the server's streams (requests that arrive
 * while others run are admitted as soon as a slot and memory free up, and
 * their kernels overlap on the device), keeps plans resident in an LRU
 * cache, and marks a ticket DONE when its completion event has fired.
 * Results do not depend on the mix: every request runs the same kernels on
 * its own workspace, with no cross-request reduction.  Policy 0 (default):
 * requests of estimated work grid points x (5 for FP64) >= 4e7 (a 384^3 FP32
 * or 256^3 FP64 solve and larger) go to a bulk lane of low-priority streams
 * (a quarter of them, at least one) and launch one CTA per tile, the others
 * to high-priority streams; within its lane a request takes the stream with
 * the least estimated work in flight, so small requests neither queue behind
 * a long solve on a stream nor wait for its persistent grids to drain.
 * Policy 1: every stream at default priority, round robin, persistent grids. */
fsa_status fsa_serve_create(fsa_server** out, const fsa_serve_opts* opts);
fsa_status fsa_serve_submit(fsa_server* s, const fsa_request* req, uint64_t* ticket);
/* Non-blocking unless timeout_s > 0: waits up to timeout_s for DONE/FAILED
 * and returns FSA_ERR_TIMEOUT if it does not come.  times may be NULL.
 * A DONE or FAILED ticket is forgotten after it has been reported. */
fsa_status fsa_serve_poll(fsa_server* s, uint64_t ticket, double timeout_s,
                          fsa_req_state* state, fsa_req_times* times);
fsa_status fsa_serve_stats_get(fsa_server* s, fsa_serve_stats* st);
/* Waits for in-flight work, then frees everything the server holds. */
fsa_status fsa_serve_destroy(fsa_server* s);

#ifdef __cplusplus
}
#endif
#endif /* FSACONV_H */
