"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle (oracle/) against something other than itself:
printed values of the paper (tests/golden/, each with its citation), closed
forms, quadrature of the defining integral, brute force, and invariants.
CPU only.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import workloads as W
from oracle import closed_forms as cf
from oracle import fsa
from tests.conftest import read_golden


# ---- Table 1 / Eq. (Fourier-Symmetric): the singular part's transform ----------

def test_What_table1_values():
    for k, eps, val in read_golden("table1_coulomb3d_What.txt"):
        got = fsa.coulomb3d_What(np.array([float(k)]), float(eps))[0]
        assert got == pytest.approx(float(val), rel=1e-15, abs=0)


@pytest.mark.parametrize("eps", [0.4, 1.0])
@pytest.mark.parametrize("k", [0.0, 0.05, 0.3, 1.0, 3.0, 10.0, 40.0])
def test_What_equals_radial_fourier_integral(k, eps):
    """Table 1's closed form equals Eq. (Fourier-Symmetric) d=3 evaluated by quadrature."""
    a = fsa.coulomb3d_What(np.array([k]), eps)[0]
    b = fsa.What_by_quadrature(k, eps)
    assert abs(a - b) <= 2e-15 * abs(b) + 1e-18


def test_What_small_k_no_cancellation():
    # expm1 form keeps full relative accuracy as k -> 0 (limit eps^2/4).
    eps = 1.0
    for k in [1e-9, 1e-6, 1e-4]:
        x = (k * eps) ** 2 / 4
        series = eps ** 2 / 4 * (1 - x / 2 + x * x / 6)
        assert fsa.coulomb3d_What(np.array([k]), eps)[0] == pytest.approx(series, rel=1e-14)


def test_Ueps_limit_and_far_field():
    eps = 0.7
    r = np.array([0.0, 1e-7, 6 * eps, 9 * eps])
    u = fsa.coulomb3d_Ueps(r, eps)
    assert u[0] == pytest.approx(1 / (2 * math.pi ** 1.5 * eps), rel=1e-15)
    assert u[1] == pytest.approx(u[0], rel=1e-12)
    # erf(r/eps) ~ 1 to 16 digits for r >= 6 eps (Sec. 1)
    assert u[2] == pytest.approx(1 / (4 * math.pi * r[2]), rel=1e-15)
    assert u[3] == pytest.approx(1 / (4 * math.pi * r[3]), rel=1e-16)


# ---- Table 1, 3-D biharmonic row -------------------------------------------------

@pytest.mark.parametrize("eps", [0.4, 1.0])
@pytest.mark.parametrize("k", [0.0, 1e-5, 0.05, 0.3, 1.0, 1.9, 2.1, 3.0, 10.0])
def test_biharmonic_What_equals_radial_fourier_integral(k, eps):
    """Table 1's biharmonic closed form (series below x = 1) equals Eq.
    (Fourier-Symmetric) d=3 of r erfc(r/eps)/(8 pi) by quadrature."""
    a = fsa.biharmonic3d_What(np.array([k]), eps)[0]
    b = fsa.What_by_quadrature_kernel(k, eps, "biharmonic3d")
    assert abs(a - b) <= 1e-14 * abs(b) + 1e-20


def test_biharmonic_What_series_meets_closed_form():
    """The two evaluations agree where both are accurate (x near 1) and the
    k = 0 value is 3 eps^4 / 32."""
    eps = 0.8
    for x in (0.7, 0.95, 0.999):
        k = 2.0 * math.sqrt(x) / eps
        direct = eps ** 4 / 16 * (math.exp(-x) * (1 + x + 2 * x * x) - 1) / (x * x)
        assert fsa.biharmonic3d_What(np.array([k]), eps)[0] == pytest.approx(direct, rel=1e-14)
    assert fsa.biharmonic3d_What(np.array([0.0]), eps)[0] == 3 * eps ** 4 / 32


def test_biharmonic_Ueps_zero_and_far_field():
    eps = 0.7
    r = np.array([0.0, 6 * eps, 9 * eps])
    u = fsa.biharmonic3d_Ueps(r, eps)
    assert u[0] == 0.0
    assert u[1] == pytest.approx(r[1] / (8 * math.pi), rel=1e-15)
    assert u[2] == pytest.approx(r[2] / (8 * math.pi), rel=1e-16)


@pytest.mark.parametrize("r", [1e-3, 0.5, 2.0, 7.0])
def test_biharmonic_closed_form_equals_radial_integral(r):
    """The non-central-chi mean form of the Gaussian's biharmonic potential
    equals the radial integral of |x - y| against the density."""
    import scipy.integrate as si
    w = math.sqrt(0.6)
    f = lambda t: t * t * math.exp(-t * t / (2 * w * w)) * ((r + t) ** 3 - abs(r - t) ** 3) / (3 * r * t)
    v, _ = si.quad(f, 0, np.inf, epsabs=0, epsrel=1e-13, limit=400)
    assert cf.biharmonic_iso_gaussian_r(1.0, w, np.array([r]))[0] == pytest.approx(v / 4, rel=1e-12)


@pytest.mark.parametrize("h,n,printed", [tuple(r) for r in read_golden("table5_biharmonic3d_iso_double.txt")])
def test_table5_biharmonic3d(h, n, printed):
    """Table 5, 3-D biharmonic (L = 12, sigma^2 = 1.2, eps = 1): the printed
    discretisation errors at h = 2, 1, 1/2 to 4 digits, round-off at 1/4."""
    d = W.paper_case1(L=12.0, sigma2=1.2, gamma3=1.0, h_over_gamma=float(h))
    assert d.n[0] == int(n)
    err = fsa.rel_error(fsa.solve(d.L, d.n, 1.0, d.rho(), kernel="biharmonic3d"),
                        cf.biharmonic_density_potential(d))
    printed = float(printed)
    if printed > 1e-10:
        assert err == pytest.approx(printed, rel=5e-4)
    else:
        assert err < 4 * printed


def test_biharmonic_fft_route_equals_brute_force():
    rng = np.random.default_rng(9)
    n, L = (6, 4, 8), (2.0, 3.0, 2.5)
    T = fsa.tensor_T(L, n, 0.5, kernel="biharmonic3d")
    rho = rng.standard_normal(n)
    assert fsa.rel_error(fsa.apply_fft(T, rho), fsa.apply_direct(T, rho)) < 1e-13


def test_biharmonic_appendix_b_bound_closed_form():
    """The App. B integral of the biharmonic U - U^eps against its closed
    form (eps^4/(8 pi)) [erfc(c) (3/16 - c^4/4) + exp(-c^2) (c^3/2 + 3c/4)/(2 sqrt(pi))],
    from integrating by parts (the library evaluates this closed form)."""
    for R0, eps in ((24.0, 1.0), (8.0, 1.0), (4.0, 0.9), (2.0, 0.5)):
        c = R0 / eps
        closed = eps ** 4 / (8 * math.pi) * (math.erfc(c) * (3 / 16 - c ** 4 / 4)
                                            + math.exp(-c * c) * (c ** 3 / 2 + 3 * c / 4) / (2 * math.sqrt(math.pi)))
        q = fsa.appendix_b_bound(R0, eps, kernel="biharmonic3d")
        assert closed == pytest.approx(q, rel=1e-9, abs=1e-300)


# ---- App. B: eps thresholds ---------------------------------------------------

def test_appendix_b_thresholds():
    for R0, c, tol in read_golden("appendix_b_thresholds.txt"):
        R0, c, tol = float(R0), float(c), float(tol)
        assert fsa.appendix_b_bound(R0, R0 / c) <= tol
        # and the printed threshold is sharp to its printed digits
        assert fsa.appendix_b_bound(R0, R0 / (c - 0.05)) > tol


# ---- Table 2: the whole scheme against the paper's printed errors -------------

@pytest.mark.parametrize("h,n,printed", [tuple(r) for r in read_golden("table2_coulomb3d_iso_double.txt")][:3])
def test_table2_iso_case1(h, n, printed):
    """Table 2, 3-D double, isotropic Case I.  At h = 1 and 1/2 the error is
    the scheme's discretisation error, so matching the printed value to 3-4
    digits pins T^(1), T^(2), the mesh, the Fourier mesh and the crop.  At
    h = 1/4 the printed value is round-off."""
    d = W.paper_case1(L=8.0, sigma2=0.8, gamma3=1.0, h_over_gamma=float(h))
    assert d.n[0] == int(n)
    err = fsa.rel_error(fsa.solve(d.L, d.n, 1.0, d.rho()), cf.density_potential(d))
    printed = float(printed)
    if printed > 1e-10:
        assert err == pytest.approx(printed, rel=5e-4)
    else:
        assert err < 4 * printed


@pytest.mark.parametrize("gamma", [1.0, 0.5, 0.25, 0.125])
def test_table2_aniso_case1(gamma):
    """Table 2, 3-D double, anisotropic Case I (L=8, sigma^2=1.2, eps=0.5,
    h = gamma/4): round-off level (printed <= 5.4e-15)."""
    rows = {float(g): float(e) for c, g, e in read_golden("table2_coulomb3d_aniso_double.txt") if c == "I"}
    d = W.paper_case1(L=8.0, sigma2=1.2, gamma3=gamma, h_over_gamma=0.25)
    err = fsa.rel_error(fsa.solve(d.L, d.n, 0.5, d.rho()), cf.density_potential(d))
    assert err < max(6e-15, 2 * rows[gamma])


@pytest.mark.slow
@pytest.mark.parametrize("gamma", [1.0, 0.125])
def test_table2_aniso_case2(gamma):
    """Table 2, Case II (L=12, sigma^2=0.8, eps=0.4, x0=(1,1,0), h=gamma/8, n=192)."""
    rows = {float(g): float(e) for c, g, e in read_golden("table2_coulomb3d_aniso_double.txt") if c == "II"}
    c = W.paper_case2(gamma3=gamma, h_over_gamma=0.125)
    err = fsa.rel_error(fsa.solve(c.L, c.n, c.eps, c.rho()), cf.case2_potential(c))
    assert err < max(5e-15, 4 * rows[gamma])


def test_spectral_convergence_then_floor():
    """Thm 1: the error falls faster than any power of h until round-off."""
    errs = []
    for h in (1.0, 0.5, 0.25):
        d = W.paper_case1(L=8.0, sigma2=0.8, h_over_gamma=h)
        errs.append(fsa.rel_error(fsa.solve(d.L, d.n, 1.0, d.rho()), cf.density_potential(d)))
    assert errs[1] < errs[0] * 1e-3 and errs[2] < 1e-14


# ---- the convolution routes ----------------------------------------------------

@pytest.mark.parametrize("n", [(4, 6, 8), (8, 8, 8), (6, 12, 4)])
def test_fft_route_equals_brute_force(n):
    """Sec. 2.3's FFT route reproduces Eq. (DiscConv) summed directly."""
    rng = np.random.default_rng(7)
    L = (3.0, 4.0, 2.5)
    T = fsa.tensor_T(L, n, 0.6)
    rho = rng.standard_normal(n)
    a = fsa.apply_fft(T, rho)
    b = fsa.apply_direct(T, rho)
    assert fsa.rel_error(a, b) < 1e-13
    pts = [(0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1), (1, 2, 3)]
    assert np.allclose(fsa.apply_direct_at(T, rho, pts), [b[p] for p in pts], rtol=1e-13, atol=0)


def test_fft_route_of_a_point_charge_is_the_shifted_tensor():
    """A unit charge at index c: Eq. (DiscConv) has one nonzero term, so the
    FFT route must return T at offsets m - c, at a corner, the opposite
    corner and the centre (a wrong pad side, crop or sign fails one)."""
    n, L = (6, 8, 10), (3.0, 4.0, 2.5)
    T = fsa.tensor_T(L, n, 0.6)
    idx = np.meshgrid(*[np.arange(nj) for nj in n], indexing="ij")
    for c in [(0, 0, 0), (5, 7, 9), (3, 4, 5), (0, 7, 2)]:
        rho = np.zeros(n)
        rho[c] = 1.0
        want = fsa.T_at(T, tuple(idx[j] - c[j] for j in range(3)))
        assert fsa.rel_error(fsa.apply_fft(T, rho), want) < 1e-14
    assert not np.any(fsa.apply_fft(T, np.zeros(n)))


def test_index_reflection_and_axis_permutation():
    """Exact symmetries of Eq. (DiscConv) with T even along each axis:
    reversing axis j of rho (i -> n_j - 1 - i) reverses axis j of phi, and
    permuting the axes of rho together with L and n permutes phi.  A
    transposed operand, a one-sided pad or crop, or an odd term in T fails."""
    n, L, eps = (6, 8, 10), (3.0, 4.0, 2.5), 0.6
    rho = np.random.default_rng(12).standard_normal(n)
    phi = fsa.solve(L, n, eps, rho)
    for ax in range(3):
        got = fsa.solve(L, n, eps, np.flip(rho, axis=ax))
        assert fsa.rel_error(got, np.flip(phi, axis=ax)) < 1e-13
    for perm in [(1, 0, 2), (2, 1, 0), (0, 2, 1), (1, 2, 0)]:
        Lp = tuple(L[a] for a in perm)
        np_ = tuple(n[a] for a in perm)
        got = fsa.solve(Lp, np_, eps, np.transpose(rho, perm))
        assert fsa.rel_error(got, np.transpose(phi, perm)) < 1e-13


def test_threaded_fft_route_equals_brute_force():
    """The threaded FFT route (scipy's FFT on several host cores, used to time
    the oracle on all cores) reproduces Eq. (DiscConv) summed directly and the
    single-threaded route, for the spectrum, T^(2) and the apply."""
    rng = np.random.default_rng(9)
    n, L, eps = (6, 8, 10), (3.0, 4.0, 2.5), 0.6
    T1 = fsa.tensor_T(L, n, eps)
    T4 = fsa.tensor_T(L, n, eps, workers=4)
    assert np.max(np.abs(T4 - T1)) <= 1e-15 * np.max(np.abs(T1))
    rho = rng.standard_normal(n)
    S1, S4 = fsa.spectrum(T1), fsa.spectrum(T1, workers=4)
    assert np.max(np.abs(S4 - S1)) <= 1e-15 * np.max(np.abs(S1))
    a = fsa.apply_spectrum(S1, rho, workers=4)
    assert fsa.rel_error(a, fsa.apply_direct(T1, rho)) < 1e-13
    assert fsa.rel_error(a, fsa.apply_spectrum(S1, rho)) < 1e-14


def test_brute_force_on_a_hand_example():
    """A 2-point case worked by hand: rho nonzero at two cells, so each output
    is T at the offsets to those two cells."""
    n, L, eps = (4, 4, 4), (2.0, 2.0, 2.0), 0.8
    T = fsa.tensor_T(L, n, eps)
    rho = np.zeros(n)
    rho[0, 0, 0] = 2.0
    rho[3, 1, 2] = -1.0
    out = fsa.apply_fft(T, rho)
    for m in [(0, 0, 0), (3, 1, 2), (2, 3, 1)]:
        want = 2.0 * T[m[0], m[1], m[2]] - 1.0 * T[(m[0] - 3) % 8, (m[1] - 1) % 8, (m[2] - 2) % 8]
        assert out[m] == pytest.approx(want, rel=1e-13, abs=1e-15)


def test_tensor_real_even_and_T2_imaginary_vanishes():
    n, L = (6, 8, 4), (3.0, 4.0, 1.0)
    T2, imag = fsa.tensor_T2(L, n, 0.5, return_imag=True)
    assert imag < 1e-15 * np.abs(T2).max()
    T = fsa.tensor_T(L, n, 0.5)
    for ax in range(3):
        m = T.shape[ax]
        idx = (-np.arange(m)) % m   # offset o -> -o (o = -n maps to itself)
        assert np.allclose(np.take(T, idx, axis=ax), T, rtol=1e-14, atol=0)
    S = np.fft.fftn(T)
    assert np.abs(S.imag).max() < 1e-12 * np.abs(S.real).max()


def test_linearity_and_translation():
    n, L, eps = (8, 8, 8), (4.0, 4.0, 4.0), 1.0
    T = fsa.tensor_T(L, n, eps)
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    lhs = fsa.apply_fft(T, 2.0 * a - 0.5 * b)
    rhs = 2.0 * fsa.apply_fft(T, a) - 0.5 * fsa.apply_fft(T, b)
    assert fsa.rel_error(lhs, rhs) < 1e-13
    # translation by whole cells: support inside the box on both sides
    r = np.zeros(n)
    r[1:4, 2:5, 1:3] = rng.standard_normal((3, 3, 2))
    s = np.roll(r, (2, 1, 3), axis=(0, 1, 2))
    pa, pb = fsa.apply_fft(T, r), fsa.apply_fft(T, s)
    assert np.allclose(np.roll(pa, (2, 1, 3), axis=(0, 1, 2))[2:, 1:, 3:], pb[2:, 1:, 3:], rtol=0, atol=1e-14)


def test_eps_independence_within_discretisation_error():
    d = W.paper_case1(L=8.0, sigma2=0.8, h_over_gamma=0.25)
    rho = d.rho()
    a = fsa.solve(d.L, d.n, 1.0, rho)
    b = fsa.solve(d.L, d.n, 1.4, rho)
    assert fsa.rel_error(a, b) < 1e-13


def test_spectrum_octant_is_whole_spectrum():
    n, L = (4, 6, 8), (2.0, 3.0, 4.0)
    T = fsa.tensor_T(L, n, 0.5)
    S = fsa.spectrum(T)
    O = fsa.spectrum_octant(T, n)
    for k in np.ndindex(*S.shape):
        p = tuple(min(k[j], S.shape[j] - k[j]) for j in range(3))
        assert S[k] == pytest.approx(O[p], rel=1e-12, abs=1e-15 * np.abs(S).max())


# ---- closed forms (the exact answers) ------------------------------------------

def test_closed_form_iso_solves_poisson():
    """-Laplacian of the erf potential reproduces the Gaussian density
    (4th-order finite differences, away from r = 0)."""
    w, hh = 0.9, 1e-2
    pts = np.array([[0.3, -0.2, 0.5], [1.1, 0.4, -0.7], [-0.5, 2.0, 0.1]])
    def phi(p):
        r = np.linalg.norm(p, axis=-1)
        return (2 * math.pi * w * w) ** 1.5 * np.vectorize(math.erf)(r / (math.sqrt(2) * w)) / (4 * math.pi * r)
    lap = 0
    for j in range(3):
        e = np.zeros(3); e[j] = hh
        lap = lap + (-phi(pts + 2 * e) + 16 * phi(pts + e) - 30 * phi(pts) + 16 * phi(pts - e) - phi(pts - 2 * e)) / (12 * hh * hh)
    rho = np.exp(-np.sum(pts ** 2, axis=1) / (2 * w * w))
    assert np.allclose(-lap, rho, rtol=1e-6, atol=1e-8)


def test_closed_form_aniso_reduces_to_iso_and_solves_poisson():
    pts = np.array([[0.0, 0.0, 0.0], [0.3, -1.2, 0.8], [3.0, 2.0, -4.0]])
    iso = cf.aniso_gaussian_potential_points(1.3, (0.1, 0.2, -0.3), (0.8, 0.8, 0.8), pts)
    r = np.linalg.norm(pts - np.array([0.1, 0.2, -0.3]), axis=1)
    q = 1.3 * (2 * math.pi * 0.64) ** 1.5
    ref = q * np.array([math.erf(x / (math.sqrt(2) * 0.8)) for x in r]) / (4 * math.pi * r)
    assert np.allclose(iso, ref, rtol=1e-14, atol=0)
    # anisotropic: finite-difference Laplacian
    sig, hh = (0.4, 0.7, 1.5), 1e-2
    p0 = np.array([[0.2, 0.1, -0.3], [0.5, -0.6, 1.0]])
    f = lambda p: cf.aniso_gaussian_potential_points(1.0, (0, 0, 0), sig, p)
    lap = 0
    for j in range(3):
        e = np.zeros(3); e[j] = hh
        lap = lap + (-f(p0 + 2 * e) + 16 * f(p0 + e) - 30 * f(p0) + 16 * f(p0 - e) - f(p0 - 2 * e)) / (12 * hh * hh)
    rho = np.exp(-np.sum(p0 ** 2 / (2 * np.array(sig) ** 2), axis=1))
    assert np.allclose(-lap, rho, rtol=1e-6, atol=1e-8)


def test_case2_density_is_minus_laplacian():
    c = W.paper_case2(L=4.0, gamma3=0.5, h_over_gamma=0.25)
    rho = c.rho()
    phi = cf.case2_potential(c)
    h = [2 * c.L[j] / c.n[j] for j in range(3)]
    lap = sum((np.roll(phi, -1, j) - 2 * phi + np.roll(phi, 1, j))[2:-2, 2:-2, 2:-2] / h[j] ** 2 for j in range(3))
    inner = rho[2:-2, 2:-2, 2:-2]
    # second-order stencil: O(h^2) agreement
    assert np.max(np.abs(-lap - inner)) < 0.05 * np.max(np.abs(inner))


# ---- d = 2: the kernels of Table 1 on the plane ---------------------------------

def _case1_2d(L, s2, h):
    from workloads import grid_axes
    n = int(round(2 * L / h))
    x = grid_axes((L, L), (n, n))
    return (L, L), (n, n), np.exp(-(x[0][:, None] ** 2 + x[1][None, :] ** 2) / s2)


@pytest.mark.parametrize("kernel", ["poisson2d", "coulomb2d", "biharmonic2d"])
@pytest.mark.parametrize("eps", [0.4, 1.0])
def test_2d_What_equals_hankel_integral(kernel, eps):
    """Table 1's 2-D closed forms equal Eq. (Fourier-Symmetric), d = 2
    (2 pi int (U - U^eps) J0(kr) r dr), by quadrature."""
    for k in [0.0, 1e-5, 0.05, 0.3, 1.0, 1.9, 2.1, 3.0, 10.0]:
        a = fsa.kernel_fns(kernel)[1](np.array([k]), eps)[0]
        b = fsa.What_by_quadrature_kernel(k, eps, kernel)
        assert abs(a - b) <= 1e-14 * abs(b) + 1e-20, (k, a, b)


@pytest.mark.parametrize("kernel", ["poisson2d", "biharmonic2d"])
def test_2d_log_Ueps_series_meets_direct(kernel):
    """ln r + E1(r^2/eps^2)/2 from its series (u < 1) against the direct sum
    near u = 1, and the r = 0 limits."""
    import scipy.special as sp
    eps = 0.8
    for u in (0.9, 0.999):
        r = math.sqrt(u) * eps
        br = math.log(r) + 0.5 * sp.exp1(u)
        want = -br / (2 * math.pi) if kernel == "poisson2d" else -(r * r) / (8 * math.pi) * (br - 1)
        assert fsa.kernel_fns(kernel)[0](np.array([r]), eps)[0] == pytest.approx(want, rel=2e-15)
    u0 = fsa.kernel_fns(kernel)[0](np.array([0.0]), eps)[0]
    if kernel == "poisson2d":
        assert u0 == pytest.approx(-(math.log(eps) - 0.5 * 0.5772156649015329) / (2 * math.pi), rel=1e-15)
    else:
        assert u0 == 0.0


def test_2d_appendix_b_thresholds():
    for kernel, R0, c, tol in read_golden("appendix_b_thresholds_2d.txt"):
        R0, c, tol = float(R0), float(c), float(tol)
        assert fsa.appendix_b_bound(R0, R0 / c, kernel) <= tol
        assert fsa.appendix_b_bound(R0, R0 / (c - 0.05), kernel) > tol


@pytest.mark.parametrize("fn,args", [
    ("coulomb2d", (0.8, [1e-3, 0.7, 2.5, 6.0])),
    ("poisson2d", (0.8, [1e-3, 0.7, 2.5, 6.0])),
])
def test_2d_closed_forms_equal_radial_integrals(fn, args):
    """2-D Coulomb: the Bessel form against the angular mean of 1/|x-y| over
    a circle, (2/pi) K(m)/(r+t), m = 4rt/(r+t)^2, integrated in t.  2-D
    Poisson: the E1 form against the integral of t rho(t) ln max(r, t)."""
    import scipy.integrate as si
    import scipy.special as sp
    s2, rs = args
    for r in rs:
        if fn == "coulomb2d":
            g = lambda t: t * math.exp(-t * t / s2) * (2 / math.pi) * sp.ellipk(min(4 * r * t / (r + t) ** 2, 1 - 1e-16)) / (r + t)
            want = cf.coulomb2d_gaussian_r(1.0, s2, np.array([r]))[0]
        else:
            g = lambda t: -t * math.exp(-t * t / s2) * math.log(max(r, t))
            want = cf.poisson2d_gaussian_r(1.0, s2, np.array([r]))[0]
        v = si.quad(g, 0, r, limit=400, epsabs=0, epsrel=1e-12)[0] + si.quad(g, r, np.inf, limit=400, epsabs=0, epsrel=1e-12)[0]
        assert want == pytest.approx(v, rel=1e-10)


def test_2d_biharmonic_angular_mean_and_closed_form():
    """The angular mean of |x-y|^2 ln|x-y| over |y| = t used by the 2-D
    biharmonic closed form, against quadrature over the circle; and the 1-D
    integral form against a direct polar double integral at one point."""
    import scipy.integrate as si
    for r, t in ((0.7, 1.3), (2.0, 0.5), (1.0, 1.0)):
        m = si.quad(lambda th: (r * r + t * t - 2 * r * t * math.cos(th)) * 0.5
                    * math.log(r * r + t * t - 2 * r * t * math.cos(th) + 1e-300), 0, 2 * math.pi, limit=400)[0] / (2 * math.pi)
        assert m == pytest.approx((r * r + t * t) * math.log(max(r, t)) + min(r, t) ** 2, rel=1e-10)
    s2, r = 0.8, 1.1
    U = lambda s: -s * s * (math.log(s) - 1) / (8 * math.pi) if s > 0 else 0.0
    val = si.dblquad(lambda th, t: t * math.exp(-t * t / s2) * U(math.sqrt(max(r * r + t * t - 2 * r * t * math.cos(th), 0.0))),
                     0, 12, 0, 2 * math.pi, epsabs=1e-12, epsrel=1e-10)[0]
    assert cf.biharmonic2d_gaussian_r(1.0, s2, np.array([r]))[0] == pytest.approx(val, rel=1e-9)


def _check_table_row(err, printed):
    if printed > 1e-10:
        assert err == pytest.approx(printed, rel=5e-4)
    else:
        assert err < 4 * printed


@pytest.mark.parametrize("h,n,printed,taken", [tuple(r) for r in read_golden("table2_coulomb2d_iso_double.txt")])
def test_table2_coulomb2d(h, n, printed, taken):
    L, nn, rho = _case1_2d(8.0, 0.8, float(h))
    assert nn[0] == int(n)
    err = fsa.rel_error(fsa.solve(L, nn, 1.0, rho, kernel="coulomb2d"),
                        cf.radial_on_grid_2d(cf.coulomb2d_gaussian_r, 1.0, 0.8, L, nn))
    _check_table_row(err, float(taken))


@pytest.mark.parametrize("case,hg,printed", [tuple(r) for r in read_golden("table4_poisson2d_double.txt")])
def test_table4_poisson2d(case, hg, printed):
    from workloads import grid_axes
    hg, printed = float(hg), float(printed)
    if case == "iso":
        L, nn, rho = _case1_2d(8.0, 1.2, hg)
        exact = cf.radial_on_grid_2d(cf.poisson2d_gaussian_r, 1.0, 1.2, L, nn)
        err = fsa.rel_error(fsa.solve(L, nn, 1.0, rho, kernel="poisson2d"), exact)
    else:
        g, s2 = hg, 1.2 ** 2
        L, nn = (10.0, 10.0 * g), (160, 160)
        x = grid_axes(L, nn)
        X, Y = x[0][:, None], x[1][None, :]
        exact = np.exp(-(X ** 2 + Y ** 2 / g ** 2) / s2)
        rho = exact * (-4 * X ** 2 / s2 ** 2 - 4 * Y ** 2 / (g ** 4 * s2 ** 2) + 2 / s2 + 2 / (g ** 2 * s2))
        err = fsa.rel_error(fsa.solve(L, nn, 0.4, rho, kernel="poisson2d"), exact)
    if case == "iso":
        _check_table_row(err, printed)
    else:  # round-off level
        assert err < max(1e-15, 2 * printed)


@pytest.mark.parametrize("h,n,printed", [tuple(r) for r in read_golden("table5_biharmonic2d_iso_double.txt")])
def test_table5_biharmonic2d(h, n, printed):
    L, nn, rho = _case1_2d(12.0, 1.2, float(h))
    assert nn[0] == int(n)
    err = fsa.rel_error(fsa.solve(L, nn, 1.0, rho, kernel="biharmonic2d"),
                        cf.radial_on_grid_2d(cf.biharmonic2d_gaussian_r, 1.0, 1.2, L, nn))
    _check_table_row(err, float(printed))


@pytest.mark.parametrize("n", [(4, 6), (8, 8), (6, 12)])
@pytest.mark.parametrize("kernel", ["poisson2d", "coulomb2d", "biharmonic2d"])
def test_2d_fft_route_equals_brute_force(n, kernel):
    rng = np.random.default_rng(3)
    L = (3.0, 2.5)
    T = fsa.tensor_T(L, n, 0.6, kernel=kernel)
    rho = rng.standard_normal(n)
    assert fsa.rel_error(fsa.apply_fft(T, rho), fsa.apply_direct(T, rho)) < 1e-13


# ---- 3-D DDI (Example 4, Table 5) -------------------------------------------

DDI_S2, DDI_L = 1.2, 8.0


def _ddi_case(h):
    d = W.paper_case1(L=DDI_L, sigma2=DDI_S2, h_over_gamma=h)
    return d.L, d.n, d.rho()


@pytest.mark.parametrize("h,n,printed", [tuple(r) for r in read_golden("table5_ddi3d_double.txt")])
def test_table5_ddi3d_grid_reading(h, n, printed):
    """Table 5, 3-D DDI (L = 8, sigma^2 = 1.2, eps = 1, the printed n and m):
    the grid reading of d_n d_m rho reproduces h = 2, 1, 1/2 to the printed
    digits and reaches round-off at h = 1/4."""
    L, nn, rho = _ddi_case(float(h))
    assert nn[0] == int(n)
    err = fsa.rel_error(fsa.ddi3d_solve(L, nn, 1.0, rho, W.DDI_N, W.DDI_M, "grid"),
                        cf.ddi3d_gaussian_grid(DDI_S2, L, nn, W.DDI_N, W.DDI_M))
    _check_table_row(err, float(printed))


@pytest.mark.parametrize("h,n,printed", [tuple(r) for r in read_golden("table5_ddi3d_double.txt")])
def test_table5_ddi3d_kernel_reading(h, n, printed):
    """The kernel reading is as accurate as the printed row: round-off at
    h = 1/4 and within 10% of the printed discretisation error at h <= 1
    (the two readings differ only in the coarse-grid aliasing)."""
    L, nn, rho = _ddi_case(float(h))
    err = fsa.rel_error(fsa.ddi3d_solve(L, nn, 1.0, rho, W.DDI_N, W.DDI_M, "kernel"),
                        cf.ddi3d_gaussian_grid(DDI_S2, L, nn, W.DDI_N, W.DDI_M))
    printed = float(printed)
    if printed < 1e-10:
        assert err < 4 * printed
    else:
        assert 0.9 * printed < err < 1.1 * printed or float(h) == 2.0
        assert err < 1.1 * max(printed, 2.2087)


def test_ddi3d_nyquist_convention_matters_at_h2():
    """The printed h = 2 value fixes the Nyquist rule of the grid reading:
    with the mixed Nyquist terms of -(k.n)(k.m) dropped it is 2.30, not 2.2087."""
    L, nn, rho = _ddi_case(2.0)
    exact = cf.ddi3d_gaussian_grid(DDI_S2, L, nn, W.DDI_N, W.DDI_M)
    n = nn[0]
    k = 2 * math.pi * np.fft.fftfreq(n, d=1.0 / n) / (2 * L[0])
    k0 = k.copy()
    k0[n // 2] = 0
    nyq = k - k0
    K0 = np.meshgrid(k0, k0, k0, indexing="ij")
    NQ = np.meshgrid(nyq, nyq, nyq, indexing="ij")
    D = -sum(W.DDI_N[i] * K0[i] for i in range(3)) * sum(W.DDI_M[i] * K0[i] for i in range(3)) \
        - sum(W.DDI_N[i] * W.DDI_M[i] * NQ[i] ** 2 for i in range(3))
    drho = np.fft.ifftn(D * np.fft.fftn(rho)).real
    nm = float(np.dot(W.DDI_N, W.DDI_M))
    other = fsa.rel_error(-nm * rho - 3 * fsa.apply_fft(fsa.tensor_T(L, nn, 1.0), drho), exact)
    assert abs(other - 2.2087) > 0.05


def test_ddi3d_closed_form_far_field_is_the_kernel():
    """Far from the density the exact potential is q U(x) with Example 4's
    kernel U (q = (pi s2)^{3/2}, the total charge): erf(r/s) = 1 and
    exp(-r^2/s2) = 0 to double precision at r >= 8 s."""
    rng = np.random.default_rng(11)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    s = math.sqrt(DDI_S2)
    pts = d * rng.uniform(8 * s, 30 * s, (200, 1))
    for nv, mv in ((W.DDI_N, W.DDI_M), W.ddi_dipoles(5), ((0, 0, 1.0), (0, 0, 1.0))):
        got = cf.ddi3d_gaussian_points(DDI_S2, pts, nv, mv)
        want = (math.pi * DDI_S2) ** 1.5 * fsa.ddi3d_U(pts, nv, mv)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)


def test_ddi3d_closed_form_is_traceless():
    """sum_i Phi(n = m = e_i) = -3 rho - 3 Laplacian(Phi_C) = 0 (the Coulomb
    kernel is the Green's function of -Laplacian), everywhere including the
    series region near r = 0."""
    rng = np.random.default_rng(12)
    pts = rng.uniform(-3, 3, (500, 3))
    pts[:5] *= 1e-3
    tot = sum(cf.ddi3d_gaussian_points(DDI_S2, pts, e, e) for e in np.eye(3))
    scale = np.max(np.abs(cf.ddi3d_gaussian_points(DDI_S2, pts, np.eye(3)[0], np.eye(3)[0])))
    assert np.max(np.abs(tot)) < 1e-14 * scale


def test_ddi3d_closed_form_series_meets_closed_form():
    """The small-r series and the closed forms of the radial derivatives agree
    where they meet (u = a^2 r^2 = 1) and against central differences of
    erf(ar)/r."""
    a = 1 / math.sqrt(DDI_S2)
    for u in (0.999999, 1.000001):
        r = np.array([math.sqrt(u) / a])
        g = cf._erf_over_r_derivs(a, r)
        r2 = np.array([math.sqrt(2 - u) / a])
        g_other = cf._erf_over_r_derivs(a, r2)
        # both sides of u = 1 use different formulas; neighbouring points agree smoothly
        assert abs(g[0][0] - g_other[0][0]) < 1e-5 * abs(g[0][0])
    F = lambda r: math.erf(a * r) / r
    for r in (0.3, 0.9, 1.1, 2.0, 4.0):
        hh = 1e-3
        d1 = (-F(r + 2 * hh) + 8 * F(r + hh) - 8 * F(r - hh) + F(r - 2 * hh)) / (12 * hh)
        d2 = (-F(r + 2 * hh) + 16 * F(r + hh) - 30 * F(r) + 16 * F(r - hh) - F(r - 2 * hh)) / (12 * hh * hh)
        g1, g2 = cf._erf_over_r_derivs(a, np.array([r]))
        assert g1[0] == pytest.approx(d1 / r, rel=1e-8)
        assert g2[0] == pytest.approx((d2 - d1 / r) / r ** 2, rel=2e-5)


@pytest.mark.parametrize("shape", [(8, 6, 4), (4, 8, 6)])
def test_spectral_dnm_exact_on_trig_polynomials(shape):
    """d_n d_m of cos(k.x + phi) is -(k.n)(k.m) cos(k.x + phi) for grid
    frequencies below Nyquist; a Nyquist cosine along one axis j takes
    -n_j m_j (pi/h_j)^2 (its mixed terms vanish on the grid)."""
    rng = np.random.default_rng(4)
    P = (3.0, 5.0, 2.0)
    axes = [np.arange(N) * (Pj / N) for N, Pj in zip(shape, P)]
    X = np.meshgrid(*axes, indexing="ij")
    nv, mv = W.ddi_dipoles(9)
    for _ in range(4):
        q = [int(rng.integers(-(N // 2) + 1, N // 2)) for N in shape]
        k = [2 * math.pi * q[j] / P[j] for j in range(3)]
        ph = rng.uniform(0, 2 * math.pi)
        f = np.cos(sum(k[j] * X[j] for j in range(3)) + ph)
        want = -np.dot(k, nv) * np.dot(k, mv) * f
        np.testing.assert_allclose(fsa.spectral_dnm(f, P, nv, mv), want, atol=1e-11 * max(1, np.abs(want).max()))
    for j in range(3):
        kn = math.pi * shape[j] / P[j]
        f = np.cos(kn * X[j])
        np.testing.assert_allclose(fsa.spectral_dnm(f, P, nv, mv), -nv[j] * mv[j] * kn * kn * f, atol=1e-10 * kn * kn)


def test_ddi3d_readings_equal_brute_force():
    """Both readings as brute-force sums (Eq. DiscConv): the grid reading is
    the Coulomb sum over spectral_dnm(rho); the kernel reading is the sum
    over rho with the doubled-grid spectral derivative of T (a Fourier
    multiplier commutes with the circular convolution)."""
    rng = np.random.default_rng(21)
    n, L = (4, 6, 8), (3.0, 4.0, 2.5)
    rho = rng.standard_normal(n)
    nv, mv = W.ddi_dipoles(3)
    nm = float(np.dot(nv, mv))
    T = fsa.tensor_T(L, n, 0.6)
    want_grid = -nm * rho - 3 * fsa.apply_direct(T, fsa.spectral_dnm(rho, [2 * l for l in L], nv, mv))
    want_kernel = -nm * rho - 3 * fsa.apply_direct(fsa.spectral_dnm(T, [4 * l for l in L], nv, mv), rho)
    assert fsa.rel_error(fsa.ddi3d_solve(L, n, 0.6, rho, nv, mv, "grid"), want_grid) < 1e-13
    assert fsa.rel_error(fsa.ddi3d_solve(L, n, 0.6, rho, nv, mv, "kernel"), want_kernel) < 1e-13


# ---- Yukawa (Example 4), Gaussian-smoothed far-field split --------------------

YUK = 1.0  # lam of the tests (the paper does not print its lam)


def test_yukawa3d_Ueps_definition_equals_closed_form():
    """The oracle's U^eps (the heat-kernel integral from t = eps^2/4) against
    the erfc closed form of the Gaussian-smoothed kernel, and its far field."""
    r = np.array([0.0, 1e-3, 0.05, 0.3, 1.0, 2.5, 6.0, 15.0, 40.0])
    for eps, lam in ((1.0, 1.0), (0.6, 0.3), (1.5, 3.0)):
        a = fsa.yukawa3d_Ueps(r, eps, lam)
        b = cf.yukawa3d_smoothed_r(r, eps, lam)
        # the closed form is a difference of two positive terms: its rounding is
        # about 1e-16 times their sum over their difference (the condition kappa)
        bb = lam * eps / 2
        rp = np.where(r > 0, r, 1.0)
        t1 = np.where(r > 0, np.exp(-lam * rp) * sp.erfc(bb - rp / eps), 2 * math.exp(-bb * bb) / (math.sqrt(math.pi) * eps))
        t2 = np.where(r > 0, np.exp(lam * rp) * sp.erfc(bb + rp / eps), lam * sp.erfc(bb))
        kappa = (t1 + t2) / np.abs(t1 - t2)
        assert np.all(np.abs(a - b) <= 1e-15 * (5 + kappa) * np.abs(b)), (np.abs(a - b) / np.abs(b), kappa)
    far = np.array([12.0, 20.0])
    np.testing.assert_allclose(fsa.yukawa3d_Ueps(far, 1.0, 1.0), fsa.yukawa3d_U(far, 1.0), rtol=1e-14)


def test_yukawa_lambda_to_zero_gives_table1():
    """lam -> 0: the 3-D kernel's U^eps and W become Table 1's Coulomb row;
    the 2-D U - U^eps becomes the Poisson row's E1(r^2/eps^2)/(4 pi)."""
    r = np.array([0.2, 1.0, 3.0])
    np.testing.assert_allclose(fsa.yukawa3d_Ueps(r, 1.0, 1e-9), fsa.coulomb3d_Ueps(r, 1.0), rtol=1e-8)
    k = np.array([0.0, 0.4, 2.0, 9.0])
    np.testing.assert_allclose(fsa.yukawa_What(k, 1.0, 0.0)[1:], fsa.coulomb3d_What(k, 1.0)[1:], rtol=1e-15)
    d2 = fsa._yukawa_heat(r, 1.0, 1e-9, 2, lower=True)
    np.testing.assert_allclose(d2, sp.exp1(r * r) / (4 * math.pi), rtol=1e-8)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("k", [0.0, 0.3, 1.0, 4.0, 12.0])
def test_yukawa_What_equals_radial_fourier_integral(d, k):
    """W(k) against Eq. (Fourier-Symmetric) of U - U^eps by quadrature (d = 3:
    the closed form of U - U^eps; d = 2: its heat-kernel integral)."""
    import scipy.integrate as si
    eps, lam = 1.0, YUK
    if d == 3:
        diff = lambda r: fsa.yukawa3d_U(np.array([r]), lam)[0] - cf.yukawa3d_smoothed_r(np.array([r]), eps, lam)[0]
        f = lambda r: 4 * math.pi * diff(r) * (math.sin(k * r) / (k * r) if k * r > 1e-12 else 1.0) * r * r
        val, _ = si.quad(f, 1e-12, 14 * eps, epsabs=0, epsrel=1e-13, limit=400)
    else:
        diff = lambda r: fsa._yukawa_heat(np.array([r]), eps, lam, 2, lower=True)[0]
        f = lambda r: 2 * math.pi * diff(r) * sp.j0(k * r) * r
        val, _ = si.quad(f, 1e-12, 14 * eps, epsabs=0, epsrel=1e-12, limit=400, points=[1e-6, 1e-3, 0.5])
    assert fsa.yukawa_What(np.array([k]), eps, lam)[0] == pytest.approx(val, rel=1e-11, abs=1e-16)


def test_yukawa2d_exact_potential_by_two_routes():
    """The 2-D exact potential (Hankel quadrature) equals q exp(lam^2 s2/4)
    times the smoothed kernel at w^2 = s2 (heat-kernel integral): two
    different integrals of the same function."""
    r = np.array([0.0, 0.4, 1.3, 4.0, 9.0])
    s2, lam = 1.2, YUK
    a = cf.yukawa2d_gaussian_r(s2, lam, r)
    b = math.pi * s2 * math.exp(lam * lam * s2 / 4) * fsa.yukawa2d_Ueps(r, math.sqrt(s2), lam)
    np.testing.assert_allclose(a, b, rtol=1e-12)


@pytest.mark.parametrize("h", [1.0, 0.5, 0.25])
def test_yukawa3d_spectral_accuracy(h):
    """rho = exp(-|x|^2/1.2) on [-8,8]^3, eps = 1, lam = 1: the FSA solve
    against the exact potential converges spectrally, to round-off at h = 1/4
    (Table 5's Yukawa rows show the same behaviour for the paper's unstated
    lam and window)."""
    L, s2 = 8.0, 1.2
    d = W.paper_case1(L=L, sigma2=s2, h_over_gamma=h)
    x = W.grid_axes(d.L, d.n)
    R = np.sqrt(x[0][:, None, None] ** 2 + x[1][None, :, None] ** 2 + x[2][None, None, :] ** 2)
    err = fsa.rel_error(fsa.solve(d.L, d.n, 1.0, d.rho(), kernel=("yukawa3d", YUK)), cf.yukawa3d_gaussian_r(s2, YUK, R))
    bound = {1.0: 2e-2, 0.5: 2e-7, 0.25: 3e-15}[h]
    assert err < bound, err


@pytest.mark.parametrize("h", [1.0, 0.5, 0.25])
def test_yukawa2d_spectral_accuracy(h):
    L, s2 = 8.0, 1.2
    n = int(round(2 * L / h))
    x = W.grid_axes((L, L), (n, n))
    R = np.sqrt(x[0][:, None] ** 2 + x[1][None, :] ** 2)
    rho = np.exp(-R ** 2 / s2)
    err = fsa.rel_error(fsa.solve((L, L), (n, n), 1.0, rho, kernel=("yukawa2d", YUK)),
                        cf.yukawa2d_gaussian_r(s2, YUK, R))
    bound = {1.0: 2e-2, 0.5: 2e-7, 0.25: 3e-15}[h]
    assert err < bound, err


def test_yukawa_fft_route_equals_brute_force():
    rng = np.random.default_rng(17)
    for kernel, n, L in ((("yukawa3d", 0.7), (4, 6, 8), (3.0, 4.0, 2.5)), (("yukawa2d", 1.3), (6, 8), (3.0, 2.5))):
        T = fsa.tensor_T(L, n, 0.6, kernel=kernel)
        rho = rng.standard_normal(n)
        assert fsa.rel_error(fsa.apply_fft(T, rho), fsa.apply_direct(T, rho)) < 1e-13


def test_yukawa_appendix_b_bound_by_direct_integral():
    """The swapped-order bound against the direct integral of the closed-form
    3-D U - U^eps (and the 2-D heat-kernel difference)."""
    import scipy.integrate as si
    for R0, eps, lam in ((8.0, 1.0, 1.0), (6.0, 1.2, 0.5), (4.0, 1.0, 2.0)):
        f3 = lambda r: (fsa.yukawa3d_U(np.array([r]), lam)[0] - cf.yukawa3d_smoothed_r(np.array([r]), eps, lam)[0]) * r * r
        v3, _ = si.quad(f3, R0, R0 + 12 * eps, epsabs=0, epsrel=1e-10, limit=200)
        assert fsa.appendix_b_bound(R0, eps, kernel=("yukawa3d", lam)) == pytest.approx(v3, rel=1e-8)
        f2 = lambda r: fsa._yukawa_heat(np.array([r]), eps, lam, 2, lower=True)[0] * r
        v2, _ = si.quad(f2, R0, R0 + 12 * eps, epsabs=0, epsrel=1e-10, limit=200)
        assert fsa.appendix_b_bound(R0, eps, kernel=("yukawa2d", lam)) == pytest.approx(v2, rel=1e-8)
