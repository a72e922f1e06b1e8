"""Plant plausible mistakes in the oracle and check that its pins catch them.

Each mutation replaces one oracle function (CPU only, via monkeypatch) with a
version carrying a typical error: a dropped term, a wrong limit, a wrong
scale, a transposed operand, a wrong crop.  The compact pin suite below (the
paper's Table 2 values, the anisotropic Case I round-off level and brute
force) must fail for every one of them.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import workloads as W
from oracle import closed_forms as cf
from oracle import fsa


def pins_pass():
    # Table 2 iso Case I, h = 1 and 1/2 (printed 2.0681E-02, 2.5036E-06)
    for h, want in ((1.0, 2.0681e-2), (0.5, 2.5036e-6)):
        d = W.paper_case1(L=8.0, sigma2=0.8, h_over_gamma=h)
        e = fsa.rel_error(fsa.solve(d.L, d.n, 1.0, d.rho()), cf.density_potential(d))
        if abs(e - want) > 5e-4 * want:
            return False
    # Table 2 aniso Case I, gamma = 1/4: round-off
    d = W.paper_case1(L=8.0, sigma2=1.2, gamma3=0.25, h_over_gamma=0.25)
    if fsa.rel_error(fsa.solve(d.L, d.n, 0.5, d.rho()), cf.density_potential(d)) > 6e-15:
        return False
    # Table 5, 3-D biharmonic, h = 1 and 1/2 (printed 2.6307E-04, 1.1065E-10)
    for h, want in ((1.0, 2.6307e-4), (0.5, 1.1065e-10)):
        d = W.paper_case1(L=12.0, sigma2=1.2, h_over_gamma=h)
        e = fsa.rel_error(fsa.solve(d.L, d.n, 1.0, d.rho(), kernel="biharmonic3d"),
                          cf.biharmonic_density_potential(d))
        if abs(e - want) > 5e-4 * want:
            return False
    # brute force
    n, L = (4, 6, 8), (3.0, 4.0, 2.5)
    T = fsa.tensor_T(L, n, 0.6)
    rho = np.random.default_rng(7).standard_normal(n)
    if fsa.rel_error(fsa.apply_fft(T, rho), fsa.apply_direct(T, rho)) > 1e-13:
        return False
    return True


def test_unmutated_pins_pass():
    assert pins_pass()


def _ueps_zero_limit(r, eps):
    r = np.asarray(r, dtype=np.float64)
    return np.where(r > 0, sp.erf(r / eps) / (4 * math.pi * np.where(r > 0, r, 1)), 0.0)


def _what_no_limit(k, eps):
    k = np.asarray(k, dtype=np.float64)
    return np.where(k > 0, -np.expm1(-(k * eps) ** 2 / 4) / np.where(k > 0, k, 1) ** 2, 0.0)


def _what_sign(k, eps):
    return -fsa_orig["coulomb3d_What"](k, eps)


def _what_no_quarter(k, eps):
    return fsa_orig["coulomb3d_What"](k, 2.0 * eps)


def _ueps_erfc(r, eps):
    r = np.asarray(r, dtype=np.float64)
    return np.where(r > 0, sp.erfc(r / eps) / (4 * math.pi * np.where(r > 0, r, 1)), 0.0)


fsa_orig = {k: getattr(fsa, k) for k in ("coulomb3d_What", "coulomb3d_Ueps", "biharmonic3d_What",
                                         "biharmonic3d_Ueps", "tensor_T", "tensor_T1", "tensor_T2",
                                         "fourier_W", "apply_fft", "poisson2d_Ueps", "coulomb2d_What",
                                         "coulomb2d_Ueps", "biharmonic2d_What", "biharmonic2d_Ueps")}


def _mu_wrong_scale(L, n, eps, kernel="coulomb3d"):
    return fsa_orig["fourier_W"](tuple(2 * l for l in L), n, eps, kernel)


def _W_axes_transposed(L, n, eps, kernel="coulomb3d"):
    return fsa_orig["fourier_W"](tuple(L[::-1]), n, eps, kernel)


def _T1_no_h(L, n, eps, kernel="coulomb3d"):
    h = fsa.mesh_steps(L, n)
    return fsa_orig["tensor_T1"](L, n, eps, kernel) / (h[0] * h[1] * h[2])


def _T_no_T2(L, n, eps, kernel="coulomb3d"):
    return fsa_orig["tensor_T1"](L, n, eps, kernel)


def _T_no_T1(L, n, eps, kernel="coulomb3d"):
    return fsa_orig["tensor_T2"](L, n, eps, kernel=kernel)


def _bh_what_coefficient(k, eps):
    # Table 1's 2 k^2 eps^2 term read as k^2 eps^2
    k = np.asarray(k, dtype=np.float64)
    kk = np.where(k > 0, k, 1.0)
    v = (-8 + np.exp(-(kk * eps) ** 2 / 4) * (8 + (kk * eps) ** 2 + (kk * eps) ** 4)) / (8 * kk ** 4)
    return np.where(k > 0, v, 3 * eps ** 4 / 32)


def _bh_ueps_coulomb_scale(r, eps):
    # 1/(4 pi) instead of 1/(8 pi)
    return 2.0 * fsa_orig["biharmonic3d_Ueps"](r, eps)


def _bh_what_limit_dropped(k, eps):
    k = np.asarray(k, dtype=np.float64)
    return np.where(k > 0, fsa_orig["biharmonic3d_What"](k, eps), 0.0)


def _apply_wrong_crop(T, rho):
    n = rho.shape
    pad = np.zeros(T.shape)
    pad[: n[0], : n[1], : n[2]] = rho
    out = np.fft.ifftn(np.fft.fftn(T) * np.fft.fftn(pad)).real
    return out[1: n[0] + 1, : n[1], : n[2]].copy()


def _apply_pad_at_end(T, rho):
    n = rho.shape
    pad = np.zeros(T.shape)
    pad[-n[0]:, : n[1], : n[2]] = rho
    out = np.fft.ifftn(np.fft.fftn(T) * np.fft.fftn(pad)).real
    return out[: n[0], : n[1], : n[2]].copy()


MUTATIONS = {
    "Ueps limit at r=0 dropped": ("coulomb3d_Ueps", _ueps_zero_limit),
    "Ueps uses erfc": ("coulomb3d_Ueps", _ueps_erfc),
    "What limit at k=0 dropped": ("coulomb3d_What", _what_no_limit),
    "What sign flipped": ("coulomb3d_What", _what_sign),
    "What eps^2/4 -> eps^2": ("coulomb3d_What", _what_no_quarter),
    "Fourier mesh pi p/L": ("fourier_W", _mu_wrong_scale),
    "Fourier mesh axes transposed": ("fourier_W", _W_axes_transposed),
    "T1 without h^3": ("tensor_T1", _T1_no_h),
    "T2 dropped": ("tensor_T", _T_no_T2),
    "T1 dropped": ("tensor_T", _T_no_T1),
    "crop shifted": ("apply_fft", _apply_wrong_crop),
    "pad on the wrong side": ("apply_fft", _apply_pad_at_end),
    "biharmonic What 2k^2eps^2 -> k^2eps^2": ("biharmonic3d_What", _bh_what_coefficient),
    "biharmonic Ueps 1/(4 pi)": ("biharmonic3d_Ueps", _bh_ueps_coulomb_scale),
    "biharmonic What limit at k=0 dropped": ("biharmonic3d_What", _bh_what_limit_dropped),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(fsa, attr, fn)
    assert not pins_pass(), f"pins missed the planted mistake: {name}"


# ---- d = 2 -------------------------------------------------------------------

def pins_pass_2d():
    """The 2-D discretisation-error rows of Tables 2, 4 and 5 (h = 1 and 1/2)
    and brute force on a small plane."""
    from workloads import grid_axes
    rows = (("coulomb2d", 8.0, 0.8, cf.coulomb2d_gaussian_r, ((1.0, 1.3856e-2), (0.5, 2.9648e-6))),
            ("poisson2d", 8.0, 1.2, cf.poisson2d_gaussian_r, ((1.0, 1.3761e-3), (0.5, 5.5617e-9))),
            ("biharmonic2d", 12.0, 1.2, cf.biharmonic2d_gaussian_r, ((1.0, 2.6558e-5), (0.5, 5.8860e-12))))
    for kernel, L, s2, fn, tab in rows:
        for h, want in tab:
            n = int(round(2 * L / h))
            x = grid_axes((L, L), (n, n))
            rho = np.exp(-(x[0][:, None] ** 2 + x[1][None, :] ** 2) / s2)
            e = fsa.rel_error(fsa.solve((L, L), (n, n), 1.0, rho, kernel=kernel),
                              cf.radial_on_grid_2d(fn, 1.0, s2, (L, L), (n, n)))
            if abs(e - want) > 5e-4 * want:
                return False
    n, L = (6, 8), (3.0, 2.5)
    T = fsa.tensor_T(L, n, 0.6, kernel="poisson2d")
    rho = np.random.default_rng(3).standard_normal(n)
    return fsa.rel_error(fsa.apply_fft(T, rho), fsa.apply_direct(T, rho)) < 1e-13


def test_unmutated_2d_pins_pass():
    assert pins_pass_2d()


def _p2_full_E1(r, eps):
    # E1(r^2/eps^2) without the factor 1/2 of Eq. lnrAppr
    import scipy.special as sp
    r = np.asarray(r, dtype=np.float64)
    rr = np.where(r > 0, r, 1.0)
    return np.where(r > 0, -(np.log(rr) + sp.exp1((rr / eps) ** 2)) / (2 * math.pi), 0.0)


def _c2_what_no_half(k, eps):
    # erf(k eps) / k instead of erf(k eps / 2) / k
    return np.where(np.asarray(k) > 0, sp.erf(np.asarray(k) * eps) / np.where(np.asarray(k) > 0, k, 1.0), eps / math.sqrt(math.pi))


def _c2_ueps_3d_scale(r, eps):
    # 1/(4 pi r) instead of 1/(2 pi r)
    return 0.5 * fsa_orig["coulomb2d_Ueps"](r, eps)


def _b2_what_coefficient(k, eps):
    # Table 1's 4 k^2 eps^2 term read as 2 k^2 eps^2
    k = np.asarray(k, dtype=np.float64)
    kk = np.where(k > 0, k, 1.0)
    v = (-16 + np.exp(-(kk * eps) ** 2 / 4) * (16 + 2 * (kk * eps) ** 2 + (kk * eps) ** 4)) / (16 * kk ** 4)
    return np.where(k > 0, v, eps ** 4 / 32)


def _b2_ueps_no_minus_one(r, eps):
    # the "- 1" in the bracket dropped
    return fsa_orig["biharmonic2d_Ueps"](r, eps) - np.asarray(r, dtype=np.float64) ** 2 / (8 * math.pi)


MUTATIONS_2D = {
    "2-D Poisson Ueps with E1 instead of E1/2": ("poisson2d_Ueps", _p2_full_E1),
    "2-D Coulomb What erf(k eps)": ("coulomb2d_What", _c2_what_no_half),
    "2-D Coulomb Ueps 1/(4 pi r)": ("coulomb2d_Ueps", _c2_ueps_3d_scale),
    "2-D biharmonic What 4k^2eps^2 -> 2k^2eps^2": ("biharmonic2d_What", _b2_what_coefficient),
    "2-D biharmonic Ueps without -1": ("biharmonic2d_Ueps", _b2_ueps_no_minus_one),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS_2D))
def test_2d_pins_catch_mutation(name, monkeypatch):
    attr, fn = MUTATIONS_2D[name]
    monkeypatch.setattr(fsa, attr, fn)
    assert not pins_pass_2d(), f"pins missed the planted mistake: {name}"


# ---- 3-D DDI -----------------------------------------------------------------

def pins_pass_ddi():
    """Table 5's 3-D DDI row (grid reading, h = 2, 1, 1/2 to the printed
    digits; h = 1/4 round-off) and the kernel reading's round-off at h = 1/4."""
    s2 = 1.2
    for h, want in ((2.0, 2.2087), (1.0, 3.3668e-2), (0.5, 8.5098e-7), (0.25, None)):
        d = W.paper_case1(L=8.0, sigma2=s2, h_over_gamma=h)
        exact = cf.ddi3d_gaussian_grid(s2, d.L, d.n, W.DDI_N, W.DDI_M)
        e = fsa.rel_error(fsa.ddi3d_solve(d.L, d.n, 1.0, d.rho(), W.DDI_N, W.DDI_M, "grid"), exact)
        if (want is None and e > 3e-14) or (want is not None and abs(e - want) > 5e-4 * want):
            return False
        if h == 0.25:
            e = fsa.rel_error(fsa.ddi3d_solve(d.L, d.n, 1.0, d.rho(), W.DDI_N, W.DDI_M, "kernel"), exact)
            if e > 3e-14:
                return False
    return True


def test_unmutated_ddi_pins_pass():
    assert pins_pass_ddi()


def _dnm_double_period(F, periods, nvec, mvec):
    return fsa_orig_ddi["spectral_dnm_of_dft"](F, [2 * p for p in periods], nvec, mvec)


def _dnm_sign(F, periods, nvec, mvec):
    return -fsa_orig_ddi["spectral_dnm_of_dft"](F, periods, nvec, mvec)


def _dnm_n_twice(F, periods, nvec, mvec):
    return fsa_orig_ddi["spectral_dnm_of_dft"](F, periods, nvec, nvec)


def _dnm_nyquist_diagonal_only(F, periods, nvec, mvec):
    # mixed Nyquist terms of -(k.n)(k.m) dropped, diagonal ones kept
    k0, nq = [], []
    for N, P in zip(F.shape, periods):
        k = 2.0 * math.pi * np.fft.fftfreq(N, d=1.0 / N) / P
        z = k.copy()
        z[N // 2] = 0.0
        k0.append(z)
        nq.append(k - z)
    K0 = np.meshgrid(*k0, indexing="ij", sparse=True)
    NQ = np.meshgrid(*nq, indexing="ij", sparse=True)
    D = -sum(nvec[j] * K0[j] for j in range(3)) * sum(mvec[j] * K0[j] for j in range(3)) \
        - sum(nvec[j] * mvec[j] * NQ[j] ** 2 for j in range(3))
    return np.fft.ifftn(D * F).real


def _ddi_local_sign(L, n, eps, rho, nvec, mvec, derivative="grid"):
    nm = float(np.dot(nvec, mvec))
    return fsa_orig_ddi["ddi3d_solve"](L, n, eps, rho, nvec, mvec, derivative) + 2 * nm * rho


fsa_orig_ddi = {k: getattr(fsa, k) for k in ("spectral_dnm_of_dft", "ddi3d_solve")}

MUTATIONS_DDI = {
    "DDI derivative with twice the period": ("spectral_dnm_of_dft", _dnm_double_period),
    "DDI derivative sign": ("spectral_dnm_of_dft", _dnm_sign),
    "DDI derivative d_n d_n": ("spectral_dnm_of_dft", _dnm_n_twice),
    "DDI Nyquist mixed terms dropped": ("spectral_dnm_of_dft", _dnm_nyquist_diagonal_only),
    "DDI local term +(m.n) rho": ("ddi3d_solve", _ddi_local_sign),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS_DDI))
def test_ddi_pins_catch_mutation(name, monkeypatch):
    attr, fn = MUTATIONS_DDI[name]
    monkeypatch.setattr(fsa, attr, fn)
    assert not pins_pass_ddi(), f"pins missed the planted mistake: {name}"


# ---- Yukawa (Gaussian-smoothed split) ----------------------------------------

def pins_pass_yukawa():
    """Spectral accuracy to round-off at h = 1/4 (3-D and 2-D, lam = 1), and the
    3-D U^eps against its erfc closed form."""
    from workloads import grid_axes
    r = np.array([0.5, 1.0, 2.0, 4.0])
    if np.max(np.abs(fsa.yukawa3d_Ueps(r, 1.0, 1.0) / cf.yukawa3d_smoothed_r(r, 1.0, 1.0) - 1)) > 1e-13:
        return False
    L, s2, h = 8.0, 1.2, 0.25
    n = int(round(2 * L / h))
    d = W.paper_case1(L=L, sigma2=s2, h_over_gamma=h)
    x = grid_axes(d.L, d.n)
    R = np.sqrt(x[0][:, None, None] ** 2 + x[1][None, :, None] ** 2 + x[2][None, None, :] ** 2)
    if fsa.rel_error(fsa.solve(d.L, d.n, 1.0, d.rho(), kernel=("yukawa3d", 1.0)), cf.yukawa3d_gaussian_r(s2, 1.0, R)) > 3e-15:
        return False
    x2 = grid_axes((L, L), (n, n))
    R2 = np.sqrt(x2[0][:, None] ** 2 + x2[1][None, :] ** 2)
    e2 = fsa.rel_error(fsa.solve((L, L), (n, n), 1.0, np.exp(-R2 ** 2 / s2), kernel=("yukawa2d", 1.0)),
                       cf.yukawa2d_gaussian_r(s2, 1.0, R2))
    return e2 < 3e-15


def test_unmutated_yukawa_pins_pass():
    assert pins_pass_yukawa()


_yuk_orig = {k: getattr(fsa, k) for k in ("yukawa_What", "_yukawa_heat")}


def _yuk_what_no_lambda(k, eps, lam=1.0):
    return fsa_orig["coulomb3d_What"](k, eps)


def _yuk_what_lambda_only_in_denominator(k, eps, lam=1.0):
    k2 = np.asarray(k, dtype=np.float64) ** 2
    return -np.expm1(-k2 * eps * eps / 4.0) / (k2 + lam * lam)


def _yuk_heat_lower_eps2(r, eps, lam, d, lower):
    return _yuk_orig["_yukawa_heat"](r, 2.0 * eps, lam, d, lower)


def _yuk_heat_wrong_dimension(r, eps, lam, d, lower):
    return _yuk_orig["_yukawa_heat"](r, eps, lam, 5 - d, lower) * (4 * math.pi * eps * eps / 4) ** ((5 - 2 * d) / 2)


MUTATIONS_YUK = {
    "Yukawa W without lam": ("yukawa_What", _yuk_what_no_lambda),
    "Yukawa W with lam only in the denominator": ("yukawa_What", _yuk_what_lambda_only_in_denominator),
    "Yukawa U^eps smoothed from t = eps^2 instead of eps^2/4": ("_yukawa_heat", _yuk_heat_lower_eps2),
    "Yukawa heat kernel of the other dimension": ("_yukawa_heat", _yuk_heat_wrong_dimension),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS_YUK))
def test_yukawa_pins_catch_mutation(name, monkeypatch):
    attr, fn = MUTATIONS_YUK[name]
    monkeypatch.setattr(fsa, attr, fn)
    assert not pins_pass_yukawa(), f"pins missed the planted mistake: {name}"
