// W(k) for any kernel of the library by the radial Fourier integrals of
// Sec. 2.2 (Eq. Fourier-Symmetric) with adaptive Gauss-Kronrod quadrature,
// tabulated for the device as piecewise Chebyshev series in k.
//
// W approximates the whole-space Fourier transform of U - U^eps (Eq. FouTran),
// which is radial:
//   d = 3:  W(k) = 4 pi int_0^inf (U - U^eps)(r) sin(k r) / (k r) r^2 dr
//   d = 2:  W(k) = 2 pi int_0^inf (U - U^eps)(r) J0(k r) r dr.
// The paper gives closed forms for the Table 1 kernels and suggests
// Gauss-Kronrod quadrature for the others; this module computes W that way for
// every kernel (the closed forms then pin it).  U - U^eps decays like
// erfc(r / eps) for every kernel here, so the integral stops at R = 7 eps,
// where the integrand is below 1e-21 of its size.
//
// The radial rule: the 15-point Kronrod extension of the 7-point Gauss rule
// (quad.h) on panels of [0, R] no wider than a quarter of the shortest period
// of the oscillating factor (pi / (2 k_max)), the first panel graded
// geometrically towards r = 0 (the 2-D kernels' U - U^eps has a logarithmic
// singularity there), every panel bisected until the Kronrod and Gauss values
// of the k-independent part G(r) = (U - U^eps)(r) r^(d-1) agree to 1e-19 of
// int |G|.  The nodes and weights serve every k of the table, each W(k) one
// weighted sum.
//
// The table: [0, k_max] split into panels, on each the Chebyshev series of W
// of degree 24 from its values at the 25 Chebyshev points of the first kind;
// a panel is bisected while its two highest coefficients exceed 2e-17 W(0).
// The device evaluates it by Clenshaw's recurrence (tensor_gen.cu).
#include <cmath>
#include <vector>

#include "fsa_internal.h"
#include "quad.h"

namespace fsa {
namespace {

constexpr long double kPi = 3.141592653589793238462643383279502884L;

int dim_of(fsa_kernel k) { return kernel_dim(k); }

// (1/4pi) int_{x0}^inf exp(-s - c / s) ds / s, the 2-D Yukawa kernel's
// U - U^eps (s = r^2 / (4 t) in its heat-kernel integral), with s = e^v:
// int exp(-e^v - c e^-v) dv over v in [v0, ln 51] (e^-51 < 1e-22), v0 =
// max(ln x0, ln c - 5), by 16-point Gauss-Legendre on panels of width 1
// below v = -2 and 1/8 above.
long double yukawa2d_tail(long double x0, long double c) {
  static long double gx[16], gw[16];
  static bool init = false;
  if (!init) {
    gauss_legendre(16, gx, gw);
    init = true;
  }
  const long double vhi = logl(51.0L);
  long double v0 = logl(x0);
  if (c > 0) v0 = std::max(v0, logl(c) - 5.0L);
  if (v0 >= vhi) return 0;
  long double sum = 0, a = v0;
  while (a < vhi) {
    const long double w = a < -2.0L ? 1.0L : 0.125L;
    const long double b = std::min(vhi, a + w), hw = 0.5L * (b - a), mid = 0.5L * (a + b);
    for (int i = 0; i < 16; ++i) {
      const long double v = mid + hw * gx[i];
      sum += gw[i] * hw * expl(-expl(v) - c * expl(-v));
    }
    a = b;
  }
  return sum / (4 * kPi);
}

}  // namespace

// (U - U^eps)(r) of each kernel, long double (r > 0).  The Gaussian-smoothed
// splits of Table 1 leave U erfc(r/eps) (Coulomb), r erfc(r/eps)/(8 pi)
// (3-D biharmonic), E1(r^2/eps^2)/(4 pi) (2-D Poisson), r^2 E1(r^2/eps^2)/(16 pi)
// (2-D biharmonic); the Yukawa kernels (heat-kernel split, lam) leave
// [e^{-lam r} erfc(r/eps - b) + e^{lam r} erfc(r/eps + b)] / (8 pi r),
// b = lam eps / 2 (d = 3, both terms positive), and the integral above (d = 2).
long double u_minus_ueps(fsa_kernel kernel, long double lam, long double eps, long double r) {
  const long double x = r / eps;
  switch (kernel) {
    case FSA_KERNEL_COULOMB3D:
    case FSA_KERNEL_DDI3D: return erfcl(x) / (4 * kPi * r);
    case FSA_KERNEL_BIHARMONIC3D: return r * erfcl(x) / (8 * kPi);
    case FSA_KERNEL_POISSON2D: return expint_e1(x * x) / (4 * kPi);
    case FSA_KERNEL_COULOMB2D: return erfcl(x) / (2 * kPi * r);
    case FSA_KERNEL_BIHARMONIC2D: return r * r * expint_e1(x * x) / (16 * kPi);
    case FSA_KERNEL_YUKAWA3D: {
      const long double b = 0.5L * lam * eps;
      return (expl(-lam * r) * erfcl(x - b) + expl(lam * r) * erfcl(x + b)) / (8 * kPi * r);
    }
    case FSA_KERNEL_YUKAWA2D: return yukawa2d_tail(x * x, 0.25L * lam * lam * r * r);
    default: return 0;
  }
}

// Nodes r_i and weights w_i on [0, R] (w_i includes the panel's half width),
// G_i = (U - U^eps)(r_i) r_i^(d-1), and per node the panel's Gauss weight
// (0 at Kronrod-only nodes) for error estimates.
struct RadialRule {
  std::vector<long double> r, wk, wg, G;
};

static bool radial_rule(fsa_kernel kernel, double lam, double eps, double kmax, RadialRule* out) {
  long double xk[15], wk[15], wg[15];
  if (!gauss_kronrod(7, xk, wk, wg)) return false;
  const int d = dim_of(kernel);
  const long double R = 7.0L * eps;
  long double hmax = 0.25L * eps;
  if (kmax > 0) hmax = std::min(hmax, kPi / (2.0L * kmax));
  auto Gf = [&](long double r) {
    const long double u = u_minus_ueps(kernel, lam, eps, r);
    return d == 3 ? u * r * r : u * r;
  };
  struct Panel {
    long double a, b;
    int depth;
  };
  std::vector<Panel> todo, done;
  // graded start: [0, hmax 2^-45], then [hmax 2^-(j+1), hmax 2^-j], j = 44 .. 0
  todo.push_back({0.0L, ldexpl(hmax, -45), 0});
  for (int j = 44; j >= 0; --j) todo.push_back({ldexpl(hmax, -(j + 1)), ldexpl(hmax, -j), 0});
  for (long double a = hmax; a < R; a += hmax) todo.push_back({a, std::min(R, a + hmax), 0});
  // int |G| for the tolerance: one pass of the unrefined rule
  long double scale = 0;
  for (const Panel& p : todo) {
    const long double hw = 0.5L * (p.b - p.a), mid = 0.5L * (p.a + p.b);
    long double sk = 0;
    for (int i = 0; i < 15; ++i) sk += wk[i] * fabsl(Gf(mid + hw * xk[i]));
    scale += sk * hw;
  }
  const long double tol = 1e-19L * (scale > 0 ? scale : 1.0L);
  // adaptive bisection
  std::vector<Panel> stack(todo.rbegin(), todo.rend());
  while (!stack.empty()) {
    const Panel p = stack.back();
    stack.pop_back();
    const long double hw = 0.5L * (p.b - p.a), mid = 0.5L * (p.a + p.b);
    long double sk = 0, sg = 0;
    for (int i = 0; i < 15; ++i) {
      const long double g = Gf(mid + hw * xk[i]);
      sk += wk[i] * g;
      sg += wg[i] * g;
    }
    if (fabsl(sk - sg) * hw > tol && p.depth < 40) {
      stack.push_back({mid, p.b, p.depth + 1});
      stack.push_back({p.a, mid, p.depth + 1});
      continue;
    }
    done.push_back(p);
  }
  out->r.clear();
  out->wk.clear();
  out->wg.clear();
  out->G.clear();
  for (const Panel& p : done) {
    const long double hw = 0.5L * (p.b - p.a), mid = 0.5L * (p.a + p.b);
    for (int i = 0; i < 15; ++i) {
      const long double r = mid + hw * xk[i];
      out->r.push_back(r);
      out->wk.push_back(wk[i] * hw);
      out->wg.push_back(wg[i] * hw);
      out->G.push_back(Gf(r));
    }
  }
  return true;
}

// W(k) from a rule; *err (may be NULL) = |Kronrod - Gauss| summed over the panels
static long double radial_apply(const RadialRule& q, int d, long double k, long double* err) {
  long double sk = 0, sg = 0, e = 0;
  const size_t np = q.r.size() / 15;
  for (size_t p = 0; p < np; ++p) {
    long double pk = 0, pg = 0;
    for (int i = 0; i < 15; ++i) {
      const size_t j = p * 15 + i;
      const long double kr = k * q.r[j];
      long double f;
      if (d == 3) f = kr == 0 ? 1.0L : sinl(kr) / kr;
      else f = std::cyl_bessel_j(0.0L, kr);
      pk += q.wk[j] * q.G[j] * f;
      pg += q.wg[j] * q.G[j] * f;
    }
    sk += pk;
    sg += pg;
    e += fabsl(pk - pg);
  }
  if (err) *err = e * (d == 3 ? 4 * kPi : 2 * kPi);
  return sk * (d == 3 ? 4 * kPi : 2 * kPi);
}

bool radial_w_value(fsa_kernel kernel, double lam, double eps, double k, double* w, double* err) {
  RadialRule q;
  if (!radial_rule(kernel, lam, eps, k, &q)) return false;
  long double e = 0;
  *w = (double)radial_apply(q, dim_of(kernel), k, &e);
  if (err) *err = (double)e;
  return true;
}

bool radial_w_table(fsa_kernel kernel, double lam, double eps, double kmax, std::vector<double>* table,
                    int* panels) {
  RadialRule q;
  if (!radial_rule(kernel, lam, eps, kmax, &q)) return false;
  const int d = dim_of(kernel);
  constexpr int D = kWTableDegree, N = D + 1;
  const long double w0 = fabsl(radial_apply(q, d, 0, nullptr));
  const long double tol = 2e-17L * (w0 > 0 ? w0 : 1.0L);
  struct Pan {
    long double a, b;
    int depth;
  };
  std::vector<Pan> stack{{0.0L, (long double)kmax * (1 + 1e-12L) + 1e-300L, 0}}, done;
  std::vector<std::vector<long double>> coefs;
  std::vector<long double> f(N), c(N);
  while (!stack.empty()) {
    const Pan p = stack.back();
    stack.pop_back();
    for (int j = 0; j < N; ++j) {
      const long double t = cosl(kPi * (j + 0.5L) / N);
      f[j] = radial_apply(q, d, 0.5L * (p.a + p.b) + 0.5L * (p.b - p.a) * t, nullptr);
    }
    for (int m = 0; m < N; ++m) {
      long double s = 0;
      for (int j = 0; j < N; ++j) s += f[j] * cosl(kPi * m * (j + 0.5L) / N);
      c[m] = 2 * s / N;
    }
    c[0] *= 0.5L;
    if (fabsl(c[D]) + fabsl(c[D - 1]) > tol && p.depth < 20) {
      stack.push_back({0.5L * (p.a + p.b), p.b, p.depth + 1});
      stack.push_back({p.a, 0.5L * (p.a + p.b), p.depth + 1});
      continue;
    }
    done.push_back(p);
    coefs.push_back(c);
  }
  // panels come out in increasing k (left halves are processed first)
  const int P = (int)done.size();
  table->assign((size_t)(P + 1) + (size_t)P * N, 0.0);
  for (int i = 0; i < P; ++i) {
    (*table)[i] = (double)done[i].a;
    for (int m = 0; m < N; ++m) (*table)[P + 1 + (size_t)i * N + m] = (double)coefs[i][m];
  }
  (*table)[P] = (double)done[P - 1].b;
  *panels = P;
  return true;
}

}  // namespace fsa

extern "C" fsa_status fsa_radial_w(fsa_kernel kernel, double kernel_param, double eps, double k, double* w,
                                   double* err_estimate) {
  using namespace fsa;
  if (!w || !(eps > 0) || !(k >= 0) || kernel < FSA_KERNEL_COULOMB3D || kernel > FSA_KERNEL_YUKAWA2D)
    return set_error(FSA_ERR_INVALID_ARG, "fsa_radial_w: bad arguments");
  const bool yuk = kernel == FSA_KERNEL_YUKAWA3D || kernel == FSA_KERNEL_YUKAWA2D;
  const double lam = yuk ? (kernel_param > 0 ? kernel_param : 1.0) : 0.0;
  if (!radial_w_value(kernel, lam, eps, k, w, err_estimate))
    return set_error(FSA_ERR_CUDA, "fsa_radial_w: quadrature setup failed");
  return FSA_OK;
}

extern "C" fsa_status fsa_gauss_kronrod15(double* nodes, double* kronrod_weights, double* gauss_weights) {
  using namespace fsa;
  long double x[15], wk[15], wg[15];
  if (!nodes || !kronrod_weights || !gauss_weights)
    return set_error(FSA_ERR_INVALID_ARG, "fsa_gauss_kronrod15: NULL argument");
  if (!gauss_kronrod(7, x, wk, wg)) return set_error(FSA_ERR_CUDA, "fsa_gauss_kronrod15: construction failed");
  for (int i = 0; i < 15; ++i) {
    nodes[i] = (double)x[i];
    kronrod_weights[i] = (double)wk[i];
    gauss_weights[i] = (double)wg[i];
  }
  return FSA_OK;
}
