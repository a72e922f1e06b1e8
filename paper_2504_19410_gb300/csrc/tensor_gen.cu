// Tensor generation ("Precomp" of Sec. 5, Example 2), in FP64 on the device.
//
// The stored spectrum is S[p] = (DFT_{2n}(T^(1))[p] + W(|mu_p|)) / prod_j 2 n_j
// on the octant p_j in [0, n_j]:
//   * T^(1)_o = h0 h1 h2 U^eps(|o.h|) (Sec. 2.1, Eq. Tensor1; Sec. 4,
//     Eq. KerAppr; Table 1): 3-D Coulomb U^eps = erf(r/eps)/(4 pi r), with the
//     limit 1/(2 pi^{3/2} eps) at r = 0; 3-D biharmonic U^eps = r erf(r/eps)/(8 pi),
//     0 at r = 0.  T^(1) is even per axis, so its values on the octant
//     o_j in [0, n_j] define it on the doubled grid.
//   * The DFT over the doubled grid of an even sequence is a DCT-I per axis
//     (Sec. 2.3 notes the axis symmetry of T); each axis is done with the
//     library's FFT kernels on the even extension.
//   * T^(2) = iDFT(W) (Sec. 2.2, Eq. Tensor2), so its DFT is W itself, at
//     k = |mu_p|, mu_{p,j} = pi p_j / (2 L_j) (Sec. 2.4, Eq. WkAnis).  Table 1:
//     3-D Coulomb W(k) = (1 - exp(-k^2 eps^2 / 4)) / k^2, evaluated with expm1,
//     W(0) = eps^2/4; 3-D biharmonic
//     W(k) = (-8 + exp(-k^2 eps^2/4) (8 + 2 k^2 eps^2 + k^4 eps^4)) / (8 k^4)
//          = (eps^4/16) g(x), x = k^2 eps^2 / 4, g(x) = (exp(-x)(1 + x + 2x^2) - 1)/x^2,
//     summed from the Taylor series of g below x = 1 (the closed form cancels
//     there), W(0) = 3 eps^4 / 32.
//   * d = 2 (the plane kernels, Table 1): the same with two axes (the octant
//     is (n0+1) x (n1+1), the normalisation 1/(4 n0 n1)).  U^eps: Poisson
//     -(ln r + E1(r^2/eps^2)/2)/(2 pi) (Eq. lnrAppr), Coulomb erf(r/eps)/(2 pi r)
//     (limit 1/(pi^{3/2} eps)), biharmonic -r^2 (ln r + E1(r^2/eps^2)/2 - 1)/(8 pi).
//     The bracket ln r + E1(u)/2, u = r^2/eps^2, is ln eps - gamma/2 -
//     (1/2) sum_{k>=1} (-u)^k/(k k!) for u < 1 (the logarithms cancel; the E1
//     series of Abramowitz & Stegun 5.1.11) and ln r + E1(u)/2 with E1 from the
//     continued fraction of Press et al. (Numerical Recipes, expint; modified
//     Lentz) for u >= 1.  W: Poisson (1 - exp(-k^2 eps^2/4))/k^2, Coulomb
//     erf(k eps/2)/k (limit eps/sqrt(pi)), biharmonic (eps^4/16) h(x),
//     h(x) = (exp(-x)(1 + x + x^2) - 1)/x^2 from its Taylor series below x = 1.
//   * Yukawa (Example 4; lam = the plan's parameter): U^eps is U convolved with
//     the Gaussian of transform exp(-k^2 eps^2/4), i.e. the heat-kernel
//     integral int_{eps^2/4}^inf exp(-lam^2 t - r^2/(4t)) (4 pi t)^{-d/2} dt,
//     and W = (1 - exp(-(k^2 + lam^2) eps^2/4)) / (k^2 + lam^2).  d = 3, r >= eps/2:
//     the closed form (1/(8 pi r)) [exp(-lam r) erfc(b - r/eps)
//     - erfcx(b + r/eps) exp(lam r - (b + r/eps)^2)], b = lam eps / 2; otherwise
//     (d = 2 everywhere, d = 3 near r = 0 where the closed form cancels) the
//     integral in x = ln(4t/eps^2) by composite 16-point Gauss-Legendre
//     quadrature on panels of width 1/2 up to where exp(-lam^2 t) < e^-60.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fsa_internal.h"
#include "passes.cuh"
#include "quad.h"

namespace fsa {

// 16-point Gauss-Legendre rule on [-1, 1] (quad.h), set per device
__constant__ double c_gl_x[16];
__constant__ double c_gl_w[16];

// Taylor coefficients of (exp(-x)(1 + x + a x^2) - 1)/x^2 (a = 2: 3-D
// biharmonic g; a = 1: 2-D biharmonic h): the coefficient of x^m is c_{m+2},
// c_j = (-1)^j (1/j! - 1/(j-1)! + a/(j-2)!) (the exponential series times
// 1 + x + a x^2).
struct BihSeries {
  double c[30];
};
constexpr BihSeries bih_series(double a) {
  BihSeries s{};
  double f[33] = {};
  f[0] = 1.0;
  for (int i = 1; i < 33; ++i) f[i] = f[i - 1] * i;
  for (int m = 0; m < 30; ++m) {
    const int j = m + 2;
    const double sign = (j % 2 == 0) ? 1.0 : -1.0;
    s.c[m] = sign * (1.0 / f[j] - 1.0 / f[j - 1] + a / f[j - 2]);
  }
  return s;
}
__constant__ BihSeries c_bih = bih_series(2.0);
__constant__ BihSeries c_bih2 = bih_series(1.0);

// 1/(k k!) for k = 0..40 (entry 0 unused): the E1 series
struct E1Series {
  double c[41];
};
constexpr E1Series e1_series() {
  E1Series s{};
  double f = 1.0;
  for (int k = 1; k <= 40; ++k) {
    f *= k;
    s.c[k] = 1.0 / (k * f);
  }
  return s;
}
__constant__ E1Series c_e1 = e1_series();

// E1(x) for x >= 1: continued fraction (Press et al., Numerical Recipes,
// expint), evaluated by the modified Lentz method; at most 200 terms.
__device__ double e1_cfrac(double x) {
  double b = x + 1.0, c = 1.0e300, d = 1.0 / b, h = d;
  for (int i = 1; i < 200; ++i) {
    const double an = -(double)i * i;
    b += 2.0;
    d = 1.0 / (an * d + b);
    c = b + an / c;
    const double del = c * d;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  return h * exp(-x);
}

// ln(r) + E1(r^2/eps^2)/2, the bracket of Eq. lnrAppr (see the file comment)
__device__ double log_half_e1(double r, double eps) {
  const double u = (r / eps) * (r / eps);
  if (u < 1.0) {
    double acc = 0.0;
    for (int k = 40; k >= 1; --k) acc = acc * (-u) + c_e1.c[k];
    acc *= -u;
    return log(eps) - 0.5 * 0.57721566490153286060651209008240243 - 0.5 * acc;
  }
  return log(r) + 0.5 * e1_cfrac(u);
}

// Sum of c.c[m] x^m, m < 30 (Horner)
__device__ __forceinline__ double series30(const BihSeries& c, double x) {
  double g = 0.0;
#pragma unroll
  for (int m = 29; m >= 0; --m) g = g * x + c.c[m];
  return g;
}

// The Yukawa heat-kernel integral int_{eps^2/4}^inf exp(-lam^2 t - r^2/(4t))
// (4 pi t)^{-d/2} dt in x = ln(4t/eps^2) (see the file comment).
__device__ double yukawa_heat(double r, double eps, double lam, int d) {
  const double pi = 3.14159265358979323846;
  const double a = 0.25 * eps * eps, la = lam * lam * a, q = (r / eps) * (r / eps);
  // exp(-la e^x) < e^-60 beyond X; the r term only shrinks the integrand
  const double X = fmax(log(60.0 / la), 0.5);
  const int panels = (int)ceil(X / 0.5);
  const double c = d == 3 ? 1.0 / (8.0 * pi * sqrt(pi) * sqrt(a)) : 1.0 / (4.0 * pi);
  double sum = 0.0;
  for (int k = 0; k < panels; ++k) {
    const double mid = 0.5 * k + 0.25;
    double ps = 0.0;
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
      const double x = mid + 0.25 * c_gl_x[i];
      const double ex = exp(x);
      const double v = exp(-la * ex - q / ex);
      ps += c_gl_w[i] * (d == 3 ? v * exp(-0.5 * x) : v);
    }
    sum += 0.25 * ps;
  }
  return c * sum;
}

__device__ double yukawa3d_U(double r, double eps, double lam) {
  if (r < 0.5 * eps) return yukawa_heat(r, eps, lam, 3);
  const double pi = 3.14159265358979323846;
  const double b = 0.5 * lam * eps, x = b + r / eps;
  return (exp(-lam * r) * erfc(b - r / eps) - erfcx(x) * exp(lam * r - x * x)) / (8.0 * pi * r);
}

// W(k) of Table 1 at k^2 (see the file comment)
__device__ __forceinline__ double singular_W(int kernel, double k2, double e2, double lam) {
  if (kernel == FSA_KERNEL_YUKAWA3D || kernel == FSA_KERNEL_YUKAWA2D) {
    const double s = k2 + lam * lam;
    return -expm1(-0.25 * s * e2) / s;
  }
  if (kernel == FSA_KERNEL_BIHARMONIC3D || kernel == FSA_KERNEL_BIHARMONIC2D) {
    const bool d3 = kernel == FSA_KERNEL_BIHARMONIC3D;
    const double a = d3 ? 2.0 : 1.0;
    const double x = 0.25 * k2 * e2;
    const double g = x < 1.0 ? series30(d3 ? c_bih : c_bih2, x) : (exp(-x) * (1.0 + x + a * x * x) - 1.0) / (x * x);
    return e2 * e2 / 16.0 * g;
  }
  if (kernel == FSA_KERNEL_COULOMB2D) {
    const double k = sqrt(k2);
    return k > 0.0 ? erf(0.5 * k * sqrt(e2)) / k : sqrt(e2) / 1.7724538509055160272981674833411452;
  }
  return k2 > 0.0 ? -expm1(-0.25 * k2 * e2) / k2 : 0.25 * e2;  // 3-D Coulomb and 2-D Poisson
}

// U^eps of Table 1 at r
__device__ __forceinline__ double smooth_U(int kernel, double r, double eps, double lam) {
  const double pi = 3.14159265358979323846;
  switch (kernel) {
    case FSA_KERNEL_YUKAWA3D: return yukawa3d_U(r, eps, lam);
    case FSA_KERNEL_YUKAWA2D: return yukawa_heat(r, eps, lam, 2);
    case FSA_KERNEL_BIHARMONIC3D: return r * erf(r / eps) / (8.0 * pi);
    case FSA_KERNEL_POISSON2D: return -log_half_e1(r, eps) / (2.0 * pi);
    case FSA_KERNEL_COULOMB2D:
      return r > 0.0 ? erf(r / eps) / (2.0 * pi * r) : 1.0 / (5.5683279968317078453 * eps);  // 1/(pi^{3/2} eps)
    case FSA_KERNEL_BIHARMONIC2D: return -(r * r) / (8.0 * pi) * (log_half_e1(r, eps) - 1.0);
    default:
      return r > 0.0 ? erf(r / eps) / (4.0 * pi * r) : 1.0 / (2.0 * 5.5683279968317078453 * eps);
  }
}

__global__ void k_t1_octant(double* __restrict__ O, int kernel, int n0, int n1, int n2, double h0, double h1,
                            double h2, double eps, double lam) {
  const long long total = (long long)(n0 + 1) * (n1 + 1) * (n2 + 1);
  const double hv = h0 * h1 * h2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p2 = (int)(i % (n2 + 1));
    const long long r01 = i / (n2 + 1);
    const int p1 = (int)(r01 % (n1 + 1));
    const int p0 = (int)(r01 / (n1 + 1));
    const double x = p0 * h0, y = p1 * h1, z = p2 * h2;
    const double r = sqrt(x * x + y * y + z * z);
    O[i] = hv * smooth_U(kernel, r, eps, lam);
  }
}

// W(k) from the quadrature table of radial_w.cpp: the panel holding k (binary
// search over the edges), then its Chebyshev series by Clenshaw's recurrence.
__device__ double w_from_table(const double* __restrict__ tab, int P, double k) {
  constexpr int N = kWTableDegree + 1;
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  const double a = tab[lo], b = tab[lo + 1];
  const double t = fmin(1.0, fmax(-1.0, (2.0 * k - a - b) / (b - a)));
  const double* c = tab + P + 1 + (size_t)lo * N;
  double b1 = 0, b2 = 0;
  for (int m = N - 1; m >= 1; --m) {
    const double b0 = fma(2.0 * t, b1, c[m] - b2);
    b2 = b1;
    b1 = b0;
  }
  return fma(t, b1, c[0] - b2);
}

template <typename R>
__global__ void k_spectrum_finalize(const double* S1, R* S,  // may alias (FP64 plans)
                                    int kernel, int n0, int n1, int n2,
                                    double c0, double c1, double c2, double eps, double lam, double inv_norm,
                                    const double* __restrict__ wtab, int wpanels) {
  const long long total = (long long)(n0 + 1) * (n1 + 1) * (n2 + 1);
  const double e2 = eps * eps;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p2 = (int)(i % (n2 + 1));
    const long long r01 = i / (n2 + 1);
    const int p1 = (int)(r01 % (n1 + 1));
    const int p0 = (int)(r01 / (n1 + 1));
    const double m0 = c0 * p0, m1 = c1 * p1, m2 = c2 * p2;  // mu_j = pi p_j / (2 L_j)
    const double k2 = m0 * m0 + m1 * m1 + m2 * m2;
    const double w = wtab ? w_from_table(wtab, wpanels, sqrt(k2)) : singular_W(kernel, k2, e2, lam);
    S[i] = (R)((S1[i] + w) * inv_norm);
  }
}

__global__ void k_to_dw(const double* __restrict__ src, float2* __restrict__ dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const dw v = dw_from_double(src[i]);
    dst[i] = make_float2(v.hi, v.lo);
  }
}

cudaError_t spectrum_to_dw(const double* src, void* dst, size_t count, cudaStream_t s) {
  const int threads = 256;
  const int blocks = (int)std::min<long long>(((long long)count + threads - 1) / threads, 152LL * 16);
  k_to_dw<<<blocks, threads, 0, s>>>(src, (float2*)dst, (long long)count);
  return cudaGetLastError();
}

namespace {

template <int M> struct DctInst {
  using P = typename PlanFor<M>::type;
  static constexpr int W = 8;
  static constexpr int T = threads_per_line<P, W>();
  static constexpr int SM = smem_strided<P, double2, W>();
  static cudaError_t prepare() {
    return cudaFuncSetAttribute((const void*)k_dct1<P, W, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
  }
  static cudaError_t run(double* O, long long nlines, long long inner, long long os, long long is, long long es,
                         cudaStream_t s) {
    const long long pairs = (nlines + 1) / 2;
    const long long tiles = (pairs + W - 1) / W;
    k_dct1<P, W, T><<<(unsigned)tiles, W * T, SM, s>>>(O, nlines, inner, os, is, es);
    return cudaGetLastError();
  }
};

#define FSA_DCT_DISPATCH(M, CALL)                      \
  switch (M) {                                         \
    case 8: return DctInst<8>::CALL;                   \
    case 12: return DctInst<12>::CALL;                 \
    case 16: return DctInst<16>::CALL;                 \
    case 24: return DctInst<24>::CALL;                 \
    case 32: return DctInst<32>::CALL;                 \
    case 48: return DctInst<48>::CALL;                 \
    case 64: return DctInst<64>::CALL;                 \
    case 96: return DctInst<96>::CALL;                 \
    case 128: return DctInst<128>::CALL;               \
    case 192: return DctInst<192>::CALL;               \
    case 256: return DctInst<256>::CALL;               \
    case 384: return DctInst<384>::CALL;               \
    case 512: return DctInst<512>::CALL;               \
    case 768: return DctInst<768>::CALL;               \
    case 1024: return DctInst<1024>::CALL;             \
    default: break;                                    \
  }

cudaError_t dct_prepare(int M) {
  FSA_DCT_DISPATCH(M, prepare());
  return cudaErrorInvalidValue;
}

cudaError_t dct_run(int M, double* O, long long nlines, long long inner, long long os, long long is, long long es,
                    cudaStream_t s) {
  FSA_DCT_DISPATCH(M, run(O, nlines, inner, os, is, es, s));
  return cudaErrorInvalidValue;
}

#undef FSA_DCT_DISPATCH

}  // namespace

cudaError_t tensorgen_prepare(int M) { return dct_prepare(M); }

cudaError_t tensorgen_init_twiddles() {
  std::vector<double> re(kTwN), im(kTwN);
  host_twiddles(re.data(), im.data());
  std::vector<double2> t64(kTwN);
  std::vector<float2> t32(kTwN);
  for (int k = 0; k < kTwN; ++k) {
    t64[k] = make_double2(re[k], im[k]);
    t32[k] = make_float2((float)re[k], (float)im[k]);
  }
  cudaError_t e = cudaMemcpyToSymbol(g_tw64, t64.data(), sizeof(double2) * kTwN);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tw32, t32.data(), sizeof(float2) * kTwN);
  double gx[16], gw[16];
  gauss_legendre(16, gx, gw);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gl_x, gx, sizeof gx);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gl_w, gw, sizeof gw);
  return e;
}

cudaError_t tensorgen_run(fsa_kernel kernel, const int n[3], const double L[3], double eps, double lam, double* O,
                          void* out, fsa_dtype dtype, cudaStream_t s, const double* wtab, int wtab_panels) {
  // d = 2: a single plane of the octant (n2 = 0 here, unit h2), no axis-2 DCT
  const bool plane = kernel_dim(kernel) == 2;
  const int n0 = n[0], n1 = n[1], n2 = plane ? 0 : n[2];
  const long long e0 = n0 + 1, e1 = n1 + 1, e2 = n2 + 1;
  const double h0 = 2.0 * L[0] / n0, h1 = 2.0 * L[1] / n1, h2 = plane ? 1.0 : 2.0 * L[2] / n2;
  const long long total = e0 * e1 * e2;
  const int threads = 256;
  const int blocks = (int)std::min<long long>((total + threads - 1) / threads, 152LL * 16);
  k_t1_octant<<<blocks, threads, 0, s>>>(O, (int)kernel, n0, n1, n2, h0, h1, h2, eps, lam);
  cudaError_t e = cudaGetLastError();
  // axis 2: lines (p0, p1) contiguous, element stride 1
  if (e == cudaSuccess && !plane) e = dct_run(2 * n2, O, e0 * e1, e1, e1 * e2, e2, 1, s);
  // axis 1: lines (p0, p2), element stride e2
  if (e == cudaSuccess) e = dct_run(2 * n1, O, e0 * e2, e2, e1 * e2, 1, e2, s);
  // axis 0: lines (p1, p2) flattened, element stride e1 * e2
  if (e == cudaSuccess) e = dct_run(2 * n0, O, e1 * e2, e1 * e2, 0, 1, e1 * e2, s);
  if (e != cudaSuccess) return e;
  const double pi = 3.14159265358979323846;
  const double inv_norm = plane ? 1.0 / (4.0 * (double)n0 * n1) : 1.0 / (8.0 * (double)n0 * n1 * n2);
  const double c2 = plane ? 0.0 : pi / (2 * L[2]);
  if (dtype == FSA_F64)
    k_spectrum_finalize<double><<<blocks, threads, 0, s>>>(O, (double*)out, (int)kernel, n0, n1, n2, pi / (2 * L[0]),
                                                           pi / (2 * L[1]), c2, eps, lam, inv_norm, wtab,
                                                           wtab_panels);
  else
    k_spectrum_finalize<float><<<blocks, threads, 0, s>>>(O, (float*)out, (int)kernel, n0, n1, n2, pi / (2 * L[0]),
                                                          pi / (2 * L[1]), c2, eps, lam, inv_norm, wtab,
                                                          wtab_panels);
  return cudaGetLastError();
}

}  // namespace fsa
