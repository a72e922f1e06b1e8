"""The FSA convolution stated literally, in numpy FP64 (test infrastructure).

Every function follows one passage of the paper (Liu & Zhang, "Fast
convolution solver based on far-field smooth approximation",
arXiv 2504.19410).  Library primitives used as steps: numpy's FFT (or,
where a caller asks for threads, scipy's FFT of the same definition run on
several host cores; or, with fft="own", the oracle's own mixed-radix DFT in
oracle/dft.py) and scipy's erf / erfc / quad.  There is no pruning,
blocking or symmetry trick:
the convolution tensor T is built on the full doubled grid and the
convolution is a full-size complex FFT product, as Sec. 2.3 states it.

Index convention (d = 3 shown; the d = 2 kernels use the same with two
axes).  A tensor on the doubled grid has shape (2 n_0, 2 n_1,
2 n_2); entry k_j holds the offset o_j = k_j for k_j < n_j and
o_j = k_j - 2 n_j otherwise, i.e. offsets -n_j .. n_j - 1 in FFT order (the
index set I_{2N} of Sec. 2.2).  Densities and potentials are n_0 x n_1 x n_2
arrays on the mesh of Sec. 2 (x = h l, l = -n/2 .. n/2 - 1).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.integrate as si
import scipy.special as sp

from . import dft as own_dft

# ---------------------------------------------------------------- kernel ----


def coulomb3d_U(r):
    """3-D Coulomb kernel U(r) = 1/(4 pi r) (Table 1)."""
    return 1.0 / (4.0 * math.pi * r)


def coulomb3d_Ueps(r, eps):
    """Far-field smooth approximation U^eps(r) = U(r) erf(r/eps) (Sec. 4,
    Eq. KerAppr; Table 1, 3-D Coulomb row).  At r = 0 the value is the limit
    erf(r/eps)/(4 pi r) -> 1/(2 pi^{3/2} eps); the paper does not state it."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    nz = r > 0
    out[nz] = sp.erf(r[nz] / eps) / (4.0 * math.pi * r[nz])
    out[~nz] = 1.0 / (2.0 * math.pi ** 1.5 * eps)
    return out


def coulomb3d_What(k, eps):
    """Whole-space Fourier transform of U - U^eps (Table 1, 3-D Coulomb row):
    (1 - exp(-k^2 eps^2 / 4)) / k^2, written with expm1.  At k = 0 the value is
    the limit eps^2/4; the paper gives only the k != 0 form."""
    k = np.asarray(k, dtype=np.float64)
    out = np.empty_like(k)
    nz = k > 0
    out[nz] = -np.expm1(-(k[nz] * eps) ** 2 / 4.0) / k[nz] ** 2
    out[~nz] = eps * eps / 4.0
    return out


def What_by_quadrature(k, eps):
    """Eq. (Fourier-Symmetric), d = 3, evaluated by adaptive quadrature:
    4 pi int_0^inf (U - U^eps)(r) sin(kr)/(kr) r^2 dr, with
    (U - U^eps)(r) = erfc(r/eps)/(4 pi r).  Used to pin coulomb3d_What."""
    if k == 0:
        f = lambda r: sp.erfc(r / eps) * r
    else:
        f = lambda r: sp.erfc(r / eps) * math.sin(k * r) / k
    val, _ = si.quad(f, 0.0, 12.0 * eps, limit=400, epsabs=0.0, epsrel=1e-13)
    return val


def biharmonic3d_U(r):
    """3-D biharmonic kernel U(r) = r/(8 pi) (Table 1; Example 4)."""
    return r / (8.0 * math.pi)


def biharmonic3d_Ueps(r, eps):
    """Far-field smooth approximation U^eps(r) = r erf(r/eps)/(8 pi) (Table 1,
    3-D biharmonic row).  It vanishes at r = 0."""
    r = np.asarray(r, dtype=np.float64)
    return r * sp.erf(r / eps) / (8.0 * math.pi)


def biharmonic3d_What(k, eps):
    """Whole-space Fourier transform of U - U^eps (Table 1, 3-D biharmonic
    row): (-8 + exp(-k^2 eps^2/4) (8 + 2 k^2 eps^2 + k^4 eps^4)) / (8 k^4).
    With x = k^2 eps^2 / 4 this is (eps^4/16) g(x),
    g(x) = (exp(-x) (1 + x + 2 x^2) - 1) / x^2, which loses all its digits to
    cancellation as x -> 0.  For x < 1 g is summed from its Taylor series
    g(x) = sum_{j>=2} c_j x^(j-2), c_j = (-1)^j (1/j! - 1/(j-1)! + 2/(j-2)!)
    (the product of the exponential series with 1 + x + 2 x^2), 30 terms;
    g(0) = 3/2, so the k = 0 value is 3 eps^4 / 32.  The paper gives only the
    closed form."""
    k = np.asarray(k, dtype=np.float64)
    x = (k * eps) ** 2 / 4.0
    g = np.empty_like(x)
    small = x < 1.0
    xs = x[small]
    acc = np.zeros_like(xs)
    for j in range(31, 1, -1):  # Horner, highest power first
        cj = (-1) ** j * (1.0 / math.factorial(j) - 1.0 / math.factorial(j - 1) + 2.0 / math.factorial(j - 2))
        acc = acc * xs + cj
    g[small] = acc
    xl = x[~small]
    g[~small] = (np.exp(-xl) * (1.0 + xl + 2.0 * xl * xl) - 1.0) / (xl * xl)
    return eps ** 4 / 16.0 * g


# ---- 2-D kernels of Table 1 -------------------------------------------------

_EULER_GAMMA = 0.57721566490153286060651209008240243


def _log_plus_half_E1(r, eps):
    """ln(r) + E1(r^2/eps^2)/2, the bracket of the 2-D Poisson and biharmonic
    U^eps (Eq. lnrAppr).  With u = r^2/eps^2 and the series
    E1(u) = -gamma - ln(u) - sum_{k>=1} (-u)^k / (k k!) (Abramowitz & Stegun
    5.1.11) the logarithms cancel exactly:
    ln(eps) - gamma/2 - (1/2) sum_{k>=1} (-u)^k / (k k!), used for u < 1 (40
    terms); for u >= 1 the two terms are summed directly.  At r = 0 the value
    is ln(eps) - gamma/2, the limit the paper leaves implicit."""
    r = np.asarray(r, dtype=np.float64)
    u = (r / eps) ** 2
    out = np.empty_like(u)
    small = u < 1.0
    us = u[small]
    acc = np.zeros_like(us)
    for k in range(40, 0, -1):
        acc = acc * (-us) + 1.0 / (k * math.factorial(k))
    acc = acc * (-us)  # sum_{k>=1} (-u)^k / (k k!)
    out[small] = math.log(eps) - 0.5 * _EULER_GAMMA - 0.5 * acc
    ul = u[~small]
    out[~small] = np.log(r[~small]) + 0.5 * sp.exp1(ul)
    return out


def poisson2d_Ueps(r, eps):
    """2-D Poisson U^eps(r) = -(1/(2 pi)) [ln r + E1(r^2/eps^2)/2] (Eq. lnrAppr;
    Table 1); -(ln eps - gamma/2)/(2 pi) at r = 0."""
    return -_log_plus_half_E1(r, eps) / (2.0 * math.pi)


def poisson2d_What(k, eps):
    """Table 1, 2-D Poisson row: (1 - exp(-k^2 eps^2/4)) / k^2, the 3-D
    Coulomb form (limit eps^2/4)."""
    return coulomb3d_What(k, eps)


def coulomb2d_Ueps(r, eps):
    """2-D Coulomb U^eps(r) = erf(r/eps)/(2 pi r) (Table 1); limit
    1/(pi^{3/2} eps) at r = 0."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    nz = r > 0
    out[nz] = sp.erf(r[nz] / eps) / (2.0 * math.pi * r[nz])
    out[~nz] = 1.0 / (math.pi ** 1.5 * eps)
    return out


def coulomb2d_What(k, eps):
    """Table 1, 2-D Coulomb row: erf(k eps/2) / k; limit eps/sqrt(pi) at k = 0."""
    k = np.asarray(k, dtype=np.float64)
    out = np.empty_like(k)
    nz = k > 0
    out[nz] = sp.erf(k[nz] * eps / 2.0) / k[nz]
    out[~nz] = eps / math.sqrt(math.pi)
    return out


def biharmonic2d_Ueps(r, eps):
    """2-D biharmonic U^eps(r) = -(r^2/(8 pi)) [ln r + E1(r^2/eps^2)/2 - 1]
    (Table 1); 0 at r = 0."""
    r = np.asarray(r, dtype=np.float64)
    return -(r * r) / (8.0 * math.pi) * (_log_plus_half_E1(r, eps) - 1.0)


def biharmonic2d_What(k, eps):
    """Table 1, 2-D biharmonic row:
    (-16 + exp(-k^2 eps^2/4) (16 + 4 k^2 eps^2 + k^4 eps^4)) / (16 k^4)
    = (eps^4/16) h(x), x = k^2 eps^2 / 4, h(x) = (exp(-x)(1 + x + x^2) - 1)/x^2.
    For x < 1 h is summed from its Taylor series, coefficient of x^(j-2)
    (-1)^j (1/j! - 1/(j-1)! + 1/(j-2)!), 30 terms; h(0) = 1/2, so the k = 0
    value is eps^4/32."""
    k = np.asarray(k, dtype=np.float64)
    x = (k * eps) ** 2 / 4.0
    h = np.empty_like(x)
    small = x < 1.0
    xs = x[small]
    acc = np.zeros_like(xs)
    for j in range(31, 1, -1):
        cj = (-1) ** j * (1.0 / math.factorial(j) - 1.0 / math.factorial(j - 1) + 1.0 / math.factorial(j - 2))
        acc = acc * xs + cj
    h[small] = acc
    xl = x[~small]
    h[~small] = (np.exp(-xl) * (1.0 + xl + xl * xl) - 1.0) / (xl * xl)
    return eps ** 4 / 16.0 * h


# ---- Yukawa kernels (Example 4) -----------------------------------------------
# The paper gives U = exp(-lam r)/(4 pi r) (d = 3) and K0(lam r)/(2 pi) (d = 2)
# but neither lam nor the far-field approximation it used (U erf(r/eps) has a
# cusp at r = 0 here; Sec. 4 then prescribes an unspecified window).  Reading
# taken: the Gaussian-smoothed kernel, U^eps = U * g with g the Gaussian whose
# Fourier transform is exp(-k^2 eps^2/4) -- for lam = 0 exactly Table 1's
# Coulomb (d = 3) and, up to a constant, Poisson (d = 2) approximations.  From
# U(r) = int_0^inf exp(-lam^2 t) (4 pi t)^{-d/2} exp(-r^2/(4t)) dt (the heat
# kernel), U^eps is the same integral from t = eps^2/4 and U - U^eps the part
# below it, whose transform is (1 - exp(-(k^2 + lam^2) eps^2/4)) / (k^2 + lam^2).
# A kernel spec is the pair (name, lam).


def _yukawa_heat(r, eps, lam, d, lower):
    """int exp(-lam^2 t - r^2/(4t)) (4 pi t)^{-d/2} dt over t >= eps^2/4
    (lower = False: U^eps) or 0 < t < eps^2/4 (lower = True: U - U^eps), by
    adaptive quadrature in x = ln(4t/eps^2)."""
    r = np.asarray(r, dtype=np.float64)
    a = eps * eps / 4.0
    out = np.empty(r.shape)
    flat = r.ravel()
    vals = np.empty(flat.shape)
    uniq, inv = np.unique(flat, return_inverse=True)
    res = np.empty(uniq.shape)
    for i, rv in enumerate(uniq):
        def f(x, rv=rv):
            t = a * math.exp(x)
            return math.exp(-lam * lam * t - rv * rv / (4.0 * t)) * (4.0 * math.pi * t) ** (-d / 2.0) * t
        if lower:
            if rv == 0.0:  # only reachable for d = 2 at r = 0, where U is infinite
                res[i] = math.inf
                continue
            # the integrand is negligible below t = r^2 / (4 * 800)
            lo = max(-80.0, math.log(rv * rv / (4.0 * a * 800.0))) if rv > 0 else -80.0
            pts = [p for p in (math.log(rv * rv / (4.0 * a)) if rv > 0 else None,) if p is not None and lo < p < 0.0]
            res[i], _ = si.quad(f, lo, 0.0, epsabs=0.0, epsrel=2e-14, limit=400, points=pts or None)
        else:
            hi = max(60.0, math.log(800.0 / max(lam * lam * a, 1e-300)))
            hi = min(hi, 200.0)
            pts = [p for p in (math.log(rv * rv / (4.0 * a)) if rv > 0 else None,) if p is not None and 0.0 < p < hi]
            res[i], _ = si.quad(f, 0.0, hi, epsabs=0.0, epsrel=2e-14, limit=400, points=pts or None)
    vals[:] = res[inv]
    out[...] = vals.reshape(r.shape)
    return out


def yukawa3d_U(r, lam):
    """3-D Yukawa kernel exp(-lam r)/(4 pi r) (Example 4)."""
    r = np.asarray(r, dtype=np.float64)
    return np.exp(-lam * r) / (4.0 * math.pi * r)


def yukawa2d_U(r, lam):
    """2-D Yukawa kernel K0(lam r)/(2 pi) (Example 4)."""
    return sp.k0(lam * np.asarray(r, dtype=np.float64)) / (2.0 * math.pi)


def yukawa3d_Ueps(r, eps, lam=1.0):
    return _yukawa_heat(r, eps, lam, 3, lower=False)


def yukawa2d_Ueps(r, eps, lam=1.0):
    return _yukawa_heat(r, eps, lam, 2, lower=False)


def yukawa_What(k, eps, lam=1.0):
    """(1 - exp(-(k^2 + lam^2) eps^2/4)) / (k^2 + lam^2), d = 2 and 3."""
    k2 = np.asarray(k, dtype=np.float64) ** 2 + lam * lam
    return -np.expm1(-k2 * eps * eps / 4.0) / k2


# kernel name -> names of its (U^eps, What) of Table 1, looked up at call time
KERNELS = {
    "coulomb3d": ("coulomb3d_Ueps", "coulomb3d_What"),
    "biharmonic3d": ("biharmonic3d_Ueps", "biharmonic3d_What"),
    "poisson2d": ("poisson2d_Ueps", "poisson2d_What"),
    "coulomb2d": ("coulomb2d_Ueps", "coulomb2d_What"),
    "biharmonic2d": ("biharmonic2d_Ueps", "biharmonic2d_What"),
    "yukawa3d": ("yukawa3d_Ueps", "yukawa_What"),
    "yukawa2d": ("yukawa2d_Ueps", "yukawa_What"),
}
KERNEL_DIM = {"coulomb3d": 3, "biharmonic3d": 3, "poisson2d": 2, "coulomb2d": 2, "biharmonic2d": 2,
              "yukawa3d": 3, "yukawa2d": 2}


def kernel_name(kernel):
    """The name of a kernel spec (a name, or (name, parameter))."""
    return kernel[0] if isinstance(kernel, tuple) else kernel


def kernel_fns(kernel):
    """(U^eps, What) of a kernel spec: a name of Table 1, or (name, lam) for
    the Yukawa kernels."""
    if isinstance(kernel, tuple):
        name, lam = kernel
        u, w = KERNELS[name]
        fu, fw = globals()[u], globals()[w]
        return (lambda r, eps: fu(r, eps, lam)), (lambda k, eps: fw(k, eps, lam))
    u, w = KERNELS[kernel]
    return globals()[u], globals()[w]


def What_by_quadrature_kernel(k, eps, kernel):
    """Eq. (Fourier-Symmetric) by adaptive quadrature.  d = 3:
    4 pi int_0^inf (U - U^eps)(r) sin(kr)/(kr) r^2 dr with
    (U - U^eps)(r) = erfc(r/eps) / (4 pi r) (Coulomb) or r erfc(r/eps) / (8 pi)
    (biharmonic).  d = 2: 2 pi int_0^inf (U - U^eps)(r) J0(kr) r dr with
    U - U^eps = E1(r^2/eps^2)/(4 pi) (Poisson), erfc(r/eps)/(2 pi r) (Coulomb),
    r^2 E1(r^2/eps^2)/(16 pi) (biharmonic).  Pins the closed forms."""
    if kernel == "coulomb3d":
        return What_by_quadrature(k, eps)
    if kernel in ("poisson2d", "coulomb2d", "biharmonic2d"):
        diff = {"poisson2d": lambda r: sp.exp1((r / eps) ** 2) / (4.0 * math.pi),
                "coulomb2d": lambda r: sp.erfc(r / eps) / (2.0 * math.pi * r),
                "biharmonic2d": lambda r: r * r * sp.exp1((r / eps) ** 2) / (16.0 * math.pi)}[kernel]
        f = lambda r: 2.0 * math.pi * diff(r) * sp.j0(k * r) * r
        pts = [eps * 1e-6, eps * 1e-3, eps] if kernel == "poisson2d" else None
        val, _ = si.quad(f, 0.0, 12.0 * eps, limit=800, epsabs=0.0, epsrel=1e-13, points=pts)
        return val
    if k == 0:
        f = lambda r: 0.5 * sp.erfc(r / eps) * r ** 3
    else:
        f = lambda r: 0.5 * sp.erfc(r / eps) * r * r * math.sin(k * r) / k
    val, _ = si.quad(f, 0.0, 12.0 * eps, limit=400, epsabs=0.0, epsrel=1e-13)
    return val


def appendix_b_bound(R0, eps, kernel="coulomb3d"):
    """App. B: the far-field condition int_{R0}^inf |U - U^eps| r^2 dr.
    3-D Coulomb: R0^2 f(c), c = R0/eps, f(c) = (1/(4 pi c^2)) int_c^inf
    s erfc(s) ds, as App. B states it.  3-D biharmonic (App. B does not treat
    it; the same integral of its U - U^eps = r erfc(r/eps)/(8 pi)):
    (eps^4 / (8 pi)) int_c^inf s^3 erfc(s) ds.  2-D kernels: the integral
    int_{R0}^inf |U - U^eps| r dr of App. B's general bound with d = 2 (the
    paper gives its thresholds R0/5.64 for Coulomb and R0/5.75 for Poisson)."""
    c = R0 / eps
    if kernel_name(kernel) in ("yukawa3d", "yukawa2d"):
        # swapping the order: int_{R0}^inf r^{d-1} int_0^{eps^2/4} ... dt dr
        name, lam = kernel
        d = KERNEL_DIM[name]
        inner = (lambda t: math.exp(-lam * lam * t - R0 * R0 / (4 * t)) / (2 * math.pi)) if d == 2 else \
            (lambda t: math.exp(-lam * lam * t) * (4 * math.pi * t) ** -1.5 *
             (2 * t * R0 * math.exp(-R0 * R0 / (4 * t)) + math.sqrt(math.pi) * (4 * t) ** 1.5 / 4 *
              sp.erfc(R0 / (2 * math.sqrt(t)))))
        val, _ = si.quad(inner, 0.0, eps * eps / 4.0, epsabs=0.0, epsrel=1e-12, limit=200)
        return val
    if KERNEL_DIM.get(kernel) == 2:
        # d = 2: int_{R0}^inf |U - U^eps| r dr
        diff = {"poisson2d": lambda r: sp.exp1((r / eps) ** 2) / (4.0 * math.pi),
                "coulomb2d": lambda r: sp.erfc(r / eps) / (2.0 * math.pi * r),
                "biharmonic2d": lambda r: r * r * sp.exp1((r / eps) ** 2) / (16.0 * math.pi)}[kernel]
        val, _ = si.quad(lambda r: diff(r) * r, R0, np.inf, epsabs=0.0, epsrel=1e-12, limit=200)
        return val
    if kernel == "biharmonic3d":
        tail, _ = si.quad(lambda s: s ** 3 * sp.erfc(s), c, np.inf, epsabs=0.0, epsrel=1e-12, limit=200)
        return eps ** 4 * tail / (8.0 * math.pi)
    tail, _ = si.quad(lambda s: s * sp.erfc(s), c, np.inf, epsabs=0.0, epsrel=1e-12, limit=200)
    return R0 * R0 * tail / (4.0 * math.pi * c * c)


# ---------------------------------------------------------------- tensor ----


def _offsets(n):
    k = np.arange(2 * n)
    return np.where(k < n, k, k - 2 * n).astype(np.float64)


def mesh_steps(L, n):
    """h_j = 2 L_j / n_j (Sec. 2; Sec. 2.4 for the anisotropic box)."""
    return [2.0 * L[j] / n[j] for j in range(len(n))]


def _radius(axes):
    """|(x_0, ..., x_{d-1})| on the tensor grid of the given per-axis values."""
    g = np.meshgrid(*axes, indexing="ij", sparse=True)
    return np.sqrt(sum(a * a for a in g))


def tensor_T1(L, n, eps, kernel="coulomb3d"):
    """T^(1) on the doubled grid: T^(1)_o = h_0 h_1 h_2 U^eps(|(o_0 h_0, o_1 h_1,
    o_2 h_2)|) (Sec. 2.1, Eq. Tensor1; Sec. 2.4, Eq. TensorAnis first term)."""
    h = mesh_steps(L, n)
    r = _radius([_offsets(n[j]) * h[j] for j in range(len(n))])
    return float(np.prod(h)) * kernel_fns(kernel)[0](r, eps)


def fourier_W(L, n, eps, kernel="coulomb3d"):
    """W on the Fourier mesh Lambda: mu_{p,j} = pi p_j / (2 L_j),
    p_j = -n_j .. n_j - 1 (Sec. 2.2, Eqs. DisFourierSeries, Wk; Sec. 2.4,
    Eq. WkAnis), with the bounded-domain transform replaced by the whole-space
    one (Eq. FouTran), i.e. W(mu) = What(|mu|).  Stored in FFT order."""
    k = _radius([math.pi * _offsets(n[j]) / (2.0 * L[j]) for j in range(len(n))])
    return kernel_fns(kernel)[1](k, eps)


def tensor_T2(L, n, eps, return_imag=False, kernel="coulomb3d", workers=None):
    """T^(2)_o = (2N)^{-d} sum_p W(mu_p) exp(2 pi i p.o / 2N) (Sec. 2.2,
    Eq. Tensor2; Eq. TensorAnis second term): numpy's ifftn carries exactly
    this sign and normalisation.  The imaginary part vanishes in exact
    arithmetic (W is real and even); its max is returned on request."""
    T2 = _ifftn(fourier_W(L, n, eps, kernel), workers)
    if return_imag:
        return T2.real.copy(), float(np.abs(T2.imag).max())
    return T2.real.copy()


def tensor_T(L, n, eps, kernel="coulomb3d", workers=None):
    """T = T^(1) + T^(2) (Sec. 2.3, Eq. DiscConv)."""
    return tensor_T1(L, n, eps, kernel) + tensor_T2(L, n, eps, kernel=kernel, workers=workers)


def _fftn(a, workers):
    """The unnormalised forward DFT over all axes: numpy's, or with
    ``workers`` threads scipy's (the same transform, lines split over cores)."""
    if workers is None:
        return np.fft.fftn(a)
    import scipy.fft
    return scipy.fft.fftn(a, workers=workers)


def _ifftn(a, workers):
    """The inverse DFT with the 1/size normalisation, as _fftn."""
    if workers is None:
        return np.fft.ifftn(a)
    import scipy.fft
    return scipy.fft.ifftn(a, workers=workers)


def spectrum(T, workers=None):
    """DFT over the doubled grid of T, divided by prod_j 2 n_j (the inverse
    transform's normalisation), real part.  T is real and even per axis
    (Sec. 2.3), so this is real up to round-off."""
    S = _fftn(T, workers)
    return S.real / T.size


def spectrum_octant(T, n):
    """The spectrum on p_j in [0, n_j]: all of it, since it is even per axis."""
    return spectrum(T)[tuple(slice(0, nj + 1) for nj in n)].copy()


# ----------------------------------------------------------- convolution ----


def apply_fft(T, rho):
    """Phi_m = sum_i T_{m-i} rho_i (Eq. DiscConv) by the route of Sec. 2.3:
    zero-pad rho to the doubled grid, FFT, multiply by the FFT of T, inverse
    FFT, keep the first n_j entries per axis."""
    box = tuple(slice(0, nj) for nj in rho.shape)
    pad = np.zeros(T.shape)
    pad[box] = rho
    out = np.fft.ifftn(np.fft.fftn(T) * np.fft.fftn(pad))
    return out.real[box].copy()


def apply_fft_own(T, rho):
    """apply_fft with the oracle's own mixed-radix DFT (oracle/dft.py) in
    place of numpy's: the same route, checked against a transform that shares
    no code with an FFT library."""
    box = tuple(slice(0, nj) for nj in rho.shape)
    pad = np.zeros(T.shape)
    pad[box] = rho
    out = own_dft.ifftn(own_dft.fftn(T) * own_dft.fftn(pad))
    return out.real[box].copy()


def apply_spectrum(S, rho, workers=None):
    """Same as apply_fft with the spectrum of T (from ``spectrum``) cached:
    the 'Execution' phase of Example 2.  ``workers``: host threads for the
    two FFTs (None: numpy's single-threaded FFT)."""
    box = tuple(slice(0, nj) for nj in rho.shape)
    pad = np.zeros(S.shape)
    pad[box] = rho
    out = _ifftn(S * S.size * _fftn(pad, workers), workers)
    return out.real[box].copy()


def T_at(T, o):
    """T at signed offsets o = (o_0, ..., o_{d-1}) (arrays), |o_j| < n_j."""
    return T[tuple(o[j] % T.shape[j] for j in range(T.ndim))]


def apply_direct(T, rho):
    """Eq. DiscConv by brute force, O(V^2): for every output point m, the
    sum over all source points i of T_{m-i} rho_i.  Small grids only."""
    return apply_direct_at(T, rho, list(np.ndindex(*rho.shape))).reshape(rho.shape)


def apply_direct_at(T, rho, points):
    """Eq. DiscConv by brute force at selected output indices only."""
    n = rho.shape
    idx = [a.ravel() for a in np.meshgrid(*[np.arange(nj) for nj in n], indexing="ij")]
    r = rho.ravel()
    return np.array([np.dot(T_at(T, tuple(m[j] - idx[j] for j in range(len(n)))), r) for m in points])


def rel_error(a, b):
    """The error norm of Sec. 5: max|a - b| / max|b| over the grid."""
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


def solve(L, n, eps, rho, kernel="coulomb3d", fft="numpy"):
    """Tensor generation followed by the FFT route: the whole method.
    fft="own": every DFT (T^(2) = iDFT(W) included) by oracle/dft.py."""
    if fft == "own":
        T = tensor_T1(L, n, eps, kernel) + own_dft.ifftn(fourier_W(L, n, eps, kernel)).real
        return apply_fft_own(T, rho)
    return apply_fft(tensor_T(L, n, eps, kernel), rho)


# ------------------------------------ 3-D dipole-dipole interaction ----
# Sec. 5, Example 4: the 3-D DDI potential is computed through the 3-D
# Coulomb kernel, Phi = -(m.n) rho - 3 (1/(4 pi |x|)) * (d_n d_m rho),
# d_n = n . grad.  The paper does not say how d_n d_m rho is discretised; the
# printed Table 5 row (h = 2, 1, 1/2) is reproduced to all its digits by the
# spectral derivative on the computational grid ("grid" below).  The
# "kernel" reading takes the same spectral derivative on the doubled grid,
# after the convolution.

DDI_DERIVATIVES = ("grid", "kernel")


def ddi3d_U(x, nvec, mvec):
    """The 3-D DDI kernel of Example 4 at points x (shape (..., 3), x != 0):
    U(x) = (3 / (4 pi)) (m.n - 3 (x.m)(x.n) / |x|^2) / |x|^3."""
    x = np.asarray(x, dtype=np.float64)
    r2 = np.sum(x * x, axis=-1)
    xn = x @ np.asarray(nvec, dtype=np.float64)
    xm = x @ np.asarray(mvec, dtype=np.float64)
    return 3.0 / (4.0 * math.pi) * (float(np.dot(nvec, mvec)) - 3.0 * xm * xn / r2) / r2 ** 1.5


def spectral_dnm_of_dft(F, periods, nvec, mvec):
    """d_n d_m of the trigonometric interpolant of a periodic grid function
    given by its DFT F (uniform grid, period periods[j] along axis j):
    multiply F by -(k.n)(k.m) with k_j = 2 pi q_j / periods[j], q_j the
    integer DFT frequencies in numpy's order (q_j = -N_j / 2 at the Nyquist
    index), inverse DFT, real part."""
    k = [2.0 * math.pi * np.fft.fftfreq(N, d=1.0 / N) / P for N, P in zip(F.shape, periods)]
    K = np.meshgrid(*k, indexing="ij", sparse=True)
    kn = sum(nvec[j] * K[j] for j in range(F.ndim))
    km = sum(mvec[j] * K[j] for j in range(F.ndim))
    return np.fft.ifftn(-kn * km * F).real.copy()


def spectral_dnm(f, periods, nvec, mvec):
    """spectral_dnm_of_dft of the samples f."""
    return spectral_dnm_of_dft(np.fft.fftn(f), periods, nvec, mvec)


def ddi3d_solve(L, n, eps, rho, nvec, mvec, derivative="grid"):
    """The 3-D DDI potential of Example 4, the convolution with 1/(4 pi |x|)
    by FSA (tensor_T, apply_fft).
    derivative = "grid": d_n d_m rho by spectral_dnm on the computational
      grid (period 2 L_j per axis), then the Coulomb solve.
    derivative = "kernel": d_n d_m of the Coulomb convolution on the doubled
      grid, uncropped (the circular convolution of T with zero-padded rho,
      given by its DFT, the product of the DFTs), with the doubled grid's
      period 4 L_j, then the crop to the first n_j entries per axis."""
    nm = float(np.dot(nvec, mvec))
    T = tensor_T(L, n, eps)
    if derivative == "grid":
        return -nm * rho - 3.0 * apply_fft(T, spectral_dnm(rho, [2.0 * l for l in L], nvec, mvec))
    if derivative == "kernel":
        box = tuple(slice(0, nj) for nj in rho.shape)
        pad = np.zeros(T.shape)
        pad[box] = rho
        conv_dft = np.fft.fftn(T) * np.fft.fftn(pad)
        return -nm * rho - 3.0 * spectral_dnm_of_dft(conv_dft, [4.0 * l for l in L], nvec, mvec)[box]
    raise ValueError(f"unknown DDI derivative reading {derivative!r}")
