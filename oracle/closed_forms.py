"""Exact potentials of the synthetic densities: Coulomb (kernel 1/(4 pi r)) and
3-D biharmonic (kernel r/(8 pi)).

Test infrastructure.  These are not steps of the FSA method: they are the
exact answers the method approximates, derived from the densities'
definitions (the paper refers to its sources for them in Sec. 5 and does not
print them).

* Isotropic Gaussian a exp(-|x-c|^2/(2 w^2)): total charge a (2 pi w^2)^{3/2},
  potential a (2 pi w^2)^{3/2} erf(r/(sqrt2 w)) / (4 pi r), value a w^2 at r = 0.
* Anisotropic Gaussian a exp(-sum_j (x_j-c_j)^2/(2 s_j^2)): from
  1/(4 pi r) = (1/(2 pi^{3/2})) int_0^inf exp(-r^2 t^2) dt and the 1-D
  Gaussian convolution identity,
      Phi(x) = a/(2 pi^{3/2}) int_0^inf prod_j sqrt(pi/(t^2+a_j))
               exp(-a_j t^2 x_j^2/(t^2+a_j)) dt,   a_j = 1/(2 s_j^2),
  evaluated by the exp-sinh (double-exponential) trapezoid rule
  t = exp((pi/2) sinh s), step 1/32 on s in [-4.5, 4.5] (Takahashi & Mori,
  1974), which converges to ~1e-16 here (checked against adaptive quadrature).
* Example 1 Case II: rho = -Laplacian(Phi0) + shifted copy, so
  Phi = Phi0(x) + Phi0(x - x0) exactly (the Coulomb kernel is the Green's
  function of -Laplacian in 3-D).

Exact biharmonic potentials (kernel r/(8 pi), Example 4):
* Isotropic Gaussian a exp(-|x-c|^2/(2 w^2)) = q times the N(c, w^2 I)
  density, q = a (2 pi w^2)^{3/2}, so Phi(x) = q/(8 pi) E|x - c - w Z| with Z
  a standard normal 3-vector.  |x - c - w Z| / w is a non-central chi variable
  with 3 degrees of freedom and parameter lam = |x - c| / w, whose mean is
      sqrt(2/pi) exp(-lam^2/2) + (lam + 1/lam) erf(lam/sqrt2)
  (value 2 sqrt(2/pi) at lam = 0).  Pinned in the tests by the radial
  integral Phi(r) = (a/4) int_0^inf t^2 exp(-t^2/(2 w^2))
  ((r+t)^3 - |r-t|^3) / (3 r t) dt (the angular mean of |x - y| over the
  sphere |y| = t, done by hand), evaluated by quadrature.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sp

from workloads import grid_axes


def iso_gaussian_potential(amp, center, w, L, n):
    x = grid_axes(L, n)
    r = np.sqrt((x[0] - center[0])[:, None, None] ** 2 + (x[1] - center[1])[None, :, None] ** 2
                + (x[2] - center[2])[None, None, :] ** 2)
    q = amp * (2.0 * math.pi * w * w) ** 1.5
    out = np.empty_like(r)
    nz = r > 0
    out[nz] = q * sp.erf(r[nz] / (math.sqrt(2.0) * w)) / (4.0 * math.pi * r[nz])
    out[~nz] = amp * w * w
    return out


def _exp_sinh(step=1.0 / 32.0, span=4.5):
    """Nodes and weights of the exp-sinh rule on [0, inf)."""
    s = np.arange(-span, span + 0.5 * step, step)
    t = np.exp(0.5 * math.pi * np.sinh(s))
    w = step * t * 0.5 * math.pi * np.cosh(s)
    return t, w


def _axis_factor(xj, aj, t2):
    """sqrt(pi/(t^2+a)) exp(-a t^2 x^2/(t^2+a)) for x (array) against nodes t^2."""
    return (np.sqrt(math.pi / (t2 + aj))[None, :]
            * np.exp(-aj * t2[None, :] * (xj * xj)[:, None] / (t2 + aj)[None, :]))


def aniso_gaussian_potential_points(amp, center, sigma, pts):
    """Potential at physical points pts (k x 3) by the 1-D integral above."""
    t, w = _exp_sinh()
    t2 = t * t
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    val = np.ones((len(pts), len(t)))
    for j in range(3):
        val *= _axis_factor(pts[:, j] - center[j], 1.0 / (2.0 * sigma[j] ** 2), t2)
    return amp * (val @ w) / (2.0 * math.pi ** 1.5)


def aniso_gaussian_potential_grid(amp, center, sigma, L, n):
    """The same on a whole grid: the integrand factorises per axis."""
    t, w = _exp_sinh()
    t2 = t * t
    x = grid_axes(L, n)
    F = [_axis_factor(x[j] - center[j], 1.0 / (2.0 * sigma[j] ** 2), t2) for j in range(3)]
    out = np.einsum("iq,jq,kq,q->ijk", F[0], F[1], F[2], w, optimize=True)
    return amp * out / (2.0 * math.pi ** 1.5)


def density_potential(d):
    """Exact potential of a workloads.Density on its grid (sum over its terms)."""
    out = np.zeros(d.n)
    for g in d.terms:
        s = g.sigma
        if s[0] == s[1] == s[2]:
            out += iso_gaussian_potential(g.amp, g.center, s[0], d.L, d.n)
        else:
            out += aniso_gaussian_potential_grid(g.amp, g.center, s, d.L, d.n)
    return out


def density_potential_points(d, pts):
    """Exact potential of a workloads.Density at grid indices pts (k x 3 ints)."""
    pts = np.atleast_2d(pts)
    h = [2.0 * d.L[j] / d.n[j] for j in range(3)]
    xyz = np.stack([h[j] * (pts[:, j] - d.n[j] // 2) for j in range(3)], axis=1)
    out = np.zeros(len(pts))
    for g in d.terms:
        s = g.sigma
        if s[0] == s[1] == s[2]:
            r = np.sqrt(np.sum((xyz - np.array(g.center)) ** 2, axis=1))
            q = g.amp * (2.0 * math.pi * s[0] ** 2) ** 1.5
            rr = np.where(r > 0, r, 1.0)
            out += np.where(r > 0, q * sp.erf(rr / (math.sqrt(2.0) * s[0])) / (4.0 * math.pi * rr),
                            g.amp * s[0] ** 2)
        else:
            out += aniso_gaussian_potential_points(g.amp, g.center, s, xyz)
    return out


def case2_potential(c):
    """Exact potential of workloads.Case2: Phi0(x) + Phi0(x - x0)."""
    x = grid_axes(c.L, c.n)
    out = np.zeros(c.n)
    for ctr in ((0.0, 0.0, 0.0), c.x0):
        X = (x[0] - ctr[0])[:, None, None]
        Y = (x[1] - ctr[1])[None, :, None]
        Z = (x[2] - ctr[2])[None, None, :]
        out += np.exp(-(X ** 2 + Y ** 2 + Z ** 2 / c.gamma3 ** 2) / c.sigma2)
    return out


def biharmonic_iso_gaussian_r(amp, w, r):
    """Biharmonic potential of amp exp(-|x|^2/(2 w^2)) at distances r (array)."""
    r = np.asarray(r, dtype=np.float64)
    q = amp * (2.0 * math.pi * w * w) ** 1.5
    lam = r / w
    mean = np.empty_like(lam)
    nz = lam > 1e-8
    ln = lam[nz]
    mean[nz] = math.sqrt(2.0 / math.pi) * np.exp(-0.5 * ln * ln) + (ln + 1.0 / ln) * sp.erf(ln / math.sqrt(2.0))
    mean[~nz] = 2.0 * math.sqrt(2.0 / math.pi)
    return q * w * mean / (8.0 * math.pi)


def biharmonic_density_potential(d):
    """Exact biharmonic potential of a workloads.Density of isotropic terms."""
    x = grid_axes(d.L, d.n)
    out = np.zeros(d.n)
    for g in d.terms:
        s = g.sigma
        assert s[0] == s[1] == s[2], "isotropic terms only"
        r = np.sqrt((x[0] - g.center[0])[:, None, None] ** 2 + (x[1] - g.center[1])[None, :, None] ** 2
                    + (x[2] - g.center[2])[None, None, :] ** 2)
        out += biharmonic_iso_gaussian_r(g.amp, s[0], r)
    return out


# ---- 2-D kernels (Table 1), radial Gaussian rho = amp exp(-r^2/s2), s2 = sigma^2 ----

def coulomb2d_gaussian_r(amp, s2, r):
    """2-D Coulomb (1/(2 pi r)) potential of amp exp(-r^2/s2): from the
    transform pi s2 exp(-k^2 s2/4)/k and int_0^inf exp(-a k^2) J0(b k) dk =
    sqrt(pi/(4a)) exp(-b^2/(8a)) I0(b^2/(8a)):
    Phi(r) = amp (sqrt(pi s2)/2) exp(-x) I0(x), x = r^2/(2 s2)."""
    x = np.asarray(r, dtype=np.float64) ** 2 / (2.0 * s2)
    return amp * 0.5 * math.sqrt(math.pi * s2) * sp.i0e(x)


def poisson2d_gaussian_r(amp, s2, r):
    """2-D Poisson (-ln(r)/(2 pi)) potential of amp exp(-r^2/s2): the angular
    mean of ln|x - y| over |y| = t is ln max(r, t), so
    Phi(r) = -amp int_0^inf t exp(-t^2/s2) ln max(r, t) dt
           = -amp (s2/4) (2 ln r + E1(r^2/s2)),
    with 2 ln r + E1(u) = ln s2 - gamma - sum_{k>=1} (-u)^k/(k k!) for u < 1."""
    r = np.asarray(r, dtype=np.float64)
    u = r * r / s2
    br = np.empty_like(u)
    small = u < 1.0
    us = u[small]
    acc = np.zeros_like(us)
    for k in range(40, 0, -1):
        acc = acc * (-us) + 1.0 / (k * math.factorial(k))
    acc = acc * (-us)
    br[small] = math.log(s2) - 0.57721566490153286060651209008240243 - acc
    br[~small] = 2.0 * np.log(r[~small]) + sp.exp1(u[~small])
    return -amp * s2 / 4.0 * br


def biharmonic2d_gaussian_r(amp, s2, r):
    """2-D biharmonic (-r^2 (ln r - 1)/(8 pi)) potential of amp exp(-r^2/s2) by
    a 1-D integral: over the circle |y| = t the mean of |x-y|^2 is r^2 + t^2
    and that of |x-y|^2 ln|x-y| is (r^2 + t^2) ln max(r,t) + min(r,t)^2 (from
    ln|x-y| = ln R - sum_m (q^m/m) cos(m theta), q = min/max), so
    Phi(r) = -(amp/4) int_0^inf t exp(-t^2/s2) [(r^2+t^2)(ln max(r,t) - 1) + min(r,t)^2] dt,
    evaluated by adaptive quadrature split at t = r."""
    import scipy.integrate as si
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    out = np.empty_like(r)
    for i, ri in enumerate(r):
        f_in = lambda t: t * math.exp(-t * t / s2) * ((ri * ri + t * t) * (math.log(ri) - 1.0) + t * t)
        f_out = lambda t: t * math.exp(-t * t / s2) * ((ri * ri + t * t) * (math.log(t) - 1.0) + ri * ri)
        a = si.quad(f_in, 0.0, ri, epsabs=0.0, epsrel=1e-13, limit=200)[0] if ri > 0 else 0.0
        b = si.quad(f_out, ri, np.inf, epsabs=0.0, epsrel=1e-13, limit=400)[0] if ri > 0 else \
            si.quad(lambda t: t * math.exp(-t * t / s2) * t * t * (math.log(t) - 1.0), 0.0, np.inf,
                    epsabs=0.0, epsrel=1e-13, limit=400)[0]
        out[i] = -amp / 4.0 * (a + b)
    return out


def radial_on_grid_2d(fn, amp, s2, L, n):
    """A radial 2-D potential fn(amp, s2, r) on the mesh of Sec. 2 (centred
    density), evaluated once per distinct radius."""
    x = grid_axes(L, n)
    r = np.sqrt(x[0][:, None] ** 2 + x[1][None, :] ** 2)
    ru, inv = np.unique(r, return_inverse=True)
    return fn(amp, s2, ru)[inv].reshape(r.shape)


# ---- 3-D DDI (Example 4), rho = exp(-|x|^2/s2) ----------------------------

def _erf_over_r_derivs(a, r):
    """For F(r) = erf(a r) / r: g1 = F'(r)/r and g2 = (F''(r) - F'(r)/r)/r^2.
    Closed forms
        g1 = (2a/sqrt(pi)) e^{-a^2 r^2} / r^2 - erf(a r) / r^3,
        g2 = 3 erf(a r) / r^5 - (6a/sqrt(pi)) e^{-a^2 r^2} / r^4
             - (4 a^3/sqrt(pi)) e^{-a^2 r^2} / r^2,
    and for u = a^2 r^2 < 1 (where they cancel) the Maclaurin series of
    F = (2a/sqrt(pi)) sum_k c_k a^{2k} r^{2k}, c_k = (-1)^k / (k! (2k+1)):
        g1 = (2a/sqrt(pi)) a^2 sum_{k>=1} 2k c_k u^{k-1},
        g2 = (2a/sqrt(pi)) a^4 sum_{k>=2} 4k(k-1) c_k u^{k-2}."""
    r = np.asarray(r, dtype=np.float64)
    u = (a * r) ** 2
    g1 = np.empty_like(r)
    g2 = np.empty_like(r)
    small = u < 1.0
    pre = 2.0 * a / math.sqrt(math.pi)
    us = u[small]
    s1 = np.zeros_like(us)
    s2 = np.zeros_like(us)
    for k in range(40, 0, -1):
        ck = (-1) ** k / (math.factorial(k) * (2 * k + 1))
        s1 = s1 * us + 2 * k * ck
        if k >= 2:
            s2 = s2 * us + 4 * k * (k - 1) * ck
    g1[small] = pre * a * a * s1
    g2[small] = pre * a ** 4 * s2
    rl = r[~small]
    e = np.exp(-(a * rl) ** 2)
    erf = sp.erf(a * rl)
    g1[~small] = pre * e / rl ** 2 - erf / rl ** 3
    g2[~small] = 3.0 * erf / rl ** 5 - 3.0 * pre * e / rl ** 4 - 2.0 * pre * a * a * e / rl ** 2
    return g1, g2


def ddi3d_gaussian_points(s2, pts, nvec, mvec):
    """Exact 3-D DDI potential of rho = exp(-|x|^2/s2) at points pts (..., 3),
    in Example 4's reformulation Phi = -(m.n) rho - 3 d_n d_m Phi_C with the
    Coulomb potential Phi_C(r) = q erf(r/s) / (4 pi r), q = (pi s2)^{3/2}
    (the isotropic Gaussian above).  For radial Phi_C,
    d_n d_m Phi_C = (n.m) Phi_C'/r + (n.x)(m.x) (Phi_C'' - Phi_C'/r) / r^2."""
    pts = np.asarray(pts, dtype=np.float64)
    r = np.sqrt(np.sum(pts * pts, axis=-1))
    a = 1.0 / math.sqrt(s2)
    q = (math.pi * s2) ** 1.5
    g1, g2 = _erf_over_r_derivs(a, r)
    nm = float(np.dot(nvec, mvec))
    xn = pts @ np.asarray(nvec, dtype=np.float64)
    xm = pts @ np.asarray(mvec, dtype=np.float64)
    dnm = q / (4.0 * math.pi) * (nm * g1 + xn * xm * g2)
    return -nm * np.exp(-r * r / s2) - 3.0 * dnm


def ddi3d_gaussian_grid(s2, L, n, nvec, mvec):
    """ddi3d_gaussian_points on the mesh of workloads.grid_axes(L, n)."""
    x = grid_axes(L, n)
    X = np.stack(np.meshgrid(*x, indexing="ij"), axis=-1)
    return ddi3d_gaussian_points(s2, X, nvec, mvec)


# ---- Yukawa (Example 4), rho = exp(-|x|^2/s2) ----------------------------------

def yukawa3d_smoothed_r(r, w, lam):
    """The 3-D Yukawa kernel exp(-lam r)/(4 pi r) convolved with the Gaussian
    whose Fourier transform is exp(-k^2 w^2/4), in closed form (inverting
    exp(-(k^2 + lam^2) w^2/4) / (k^2 + lam^2) times exp(lam^2 w^2/4) by the
    radial sine transform):
      (1/(8 pi r)) [exp(-lam r) erfc(b - r/w) - exp(lam r) erfc(b + r/w)],
    b = lam w / 2, the second product taken as erfcx(b + r/w) exp(lam r - (b + r/w)^2);
    at r = 0: (1/(4 pi)) (2 exp(-b^2)/(sqrt(pi) w) - lam erfc(b))."""
    r = np.asarray(r, dtype=np.float64)
    b = lam * w / 2.0
    out = np.empty_like(r)
    nz = r > 0
    rr = r[nz]
    x = b + rr / w
    out[nz] = (np.exp(-lam * rr) * sp.erfc(b - rr / w) - sp.erfcx(x) * np.exp(lam * rr - x * x)) / (8.0 * math.pi * rr)
    out[~nz] = (2.0 * math.exp(-b * b) / (math.sqrt(math.pi) * w) - lam * sp.erfc(b)) / (4.0 * math.pi)
    return out


def yukawa3d_gaussian_r(s2, lam, r):
    """Exact 3-D Yukawa potential of exp(-|x|^2/s2): its transform is
    q exp(-k^2 s2/4), q = (pi s2)^{3/2}, so Phi = q exp(lam^2 s2/4) times the
    smoothed kernel with w = sqrt(s2)."""
    return (math.pi * s2) ** 1.5 * math.exp(lam * lam * s2 / 4.0) * yukawa3d_smoothed_r(r, math.sqrt(s2), lam)


def yukawa2d_gaussian_r(s2, lam, r):
    """Exact 2-D Yukawa (K0(lam r)/(2 pi)) potential of exp(-|x|^2/s2) by the
    Hankel transform: Phi(r) = (1/(2 pi)) int_0^inf pi s2 exp(-k^2 s2/4)
    J0(k r) k / (k^2 + lam^2) dk, adaptive quadrature."""
    import scipy.integrate as si
    r = np.asarray(r, dtype=np.float64)
    out = np.empty(r.shape)
    uniq, inv = np.unique(r.ravel(), return_inverse=True)
    res = np.empty(uniq.shape)
    kmax = 2.0 * math.sqrt(40.0 / s2)
    for i, rv in enumerate(uniq):
        f = lambda k: math.pi * s2 * math.exp(-k * k * s2 / 4.0) * sp.j0(k * rv) * k / (k * k + lam * lam)
        res[i], _ = si.quad(f, 0.0, kmax, epsabs=0.0, epsrel=2e-14, limit=800)
    out[...] = (res[inv] / (2.0 * math.pi)).reshape(r.shape)
    return out
