"""Pins of the oracle's own DFT (oracle/dft.py) and of the FFT route built on it.

The mixed-radix transform is checked against the DFT's definition summed as a
matrix product (brute force), against the closed-form transforms of a delta
and of a pure exponential, against Parseval's identity, and, through the whole
scheme, against the error Table 2 prints for the isotropic Case I at h = 1/2.
CPU only.
"""
import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import dft
from oracle import fsa

LENGTHS = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 16, 18, 24, 27, 32, 36, 48]


@pytest.mark.parametrize("n", LENGTHS)
@pytest.mark.parametrize("inverse", [False, True])
def test_dft_equals_definition(n, inverse):
    """Every length, forward and inverse, against the sum of the definition
    (the brute force below does not call dft_matrix: it sums j by j)."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    sign = 1.0 if inverse else -1.0
    want = np.zeros_like(x)
    for k in range(n):
        for j in range(n):
            want[:, k] += x[:, j] * np.exp(sign * 2j * np.pi * j * k / n)
    if inverse:
        want /= n
    got = dft.fft_axis(x, 1, inverse=inverse)
    assert np.abs(got - want).max() <= 1e-13 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("n", [6, 16, 24])
def test_dft_closed_forms(n):
    """DFT of a delta at j0 is exp(-2 pi i j0 k / n); DFT of exp(2 pi i q j / n)
    is n at k = q and zero elsewhere."""
    j0, q = 1, n // 3
    delta = np.zeros(n)
    delta[j0] = 1.0
    k = np.arange(n)
    assert np.allclose(dft.fft_axis(delta, 0), np.exp(-2j * np.pi * j0 * k / n), rtol=0, atol=1e-14)
    wave = np.exp(2j * np.pi * q * k / n)
    want = np.zeros(n, dtype=complex)
    want[q] = n
    assert np.allclose(dft.fft_axis(wave, 0), want, rtol=0, atol=1e-12)


def test_dft_parseval_and_roundtrip():
    """sum |x|^2 = (1/N) sum |X|^2 over a 3-D array, and ifftn(fftn(x)) = x."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((6, 8, 12))
    X = dft.fftn(x)
    assert np.sum(np.abs(X) ** 2) / x.size == pytest.approx(np.sum(x ** 2), rel=1e-13)
    assert np.abs(dft.ifftn(X) - x).max() < 1e-14


def test_dft_fftn_axes_are_independent():
    """fftn of a separable product is the product of the 1-D transforms."""
    rng = np.random.default_rng(4)
    a, b, c = rng.standard_normal(4), rng.standard_normal(6), rng.standard_normal(9)
    x = a[:, None, None] * b[None, :, None] * c[None, None, :]
    want = dft.fft_axis(a, 0)[:, None, None] * dft.fft_axis(b, 0)[None, :, None] * dft.fft_axis(c, 0)[None, None, :]
    assert np.abs(dft.fftn(x) - want).max() < 1e-12


@pytest.mark.parametrize("n", [(4, 6, 8), (6, 12, 4)])
def test_own_fft_route_equals_brute_force(n):
    """Sec. 2.3's route on the oracle's own DFT reproduces Eq. (DiscConv) summed directly."""
    rng = np.random.default_rng(7)
    L = (3.0, 4.0, 2.5)
    T = fsa.tensor_T(L, n, 0.6)
    rho = rng.standard_normal(n)
    assert fsa.rel_error(fsa.apply_fft_own(T, rho), fsa.apply_direct(T, rho)) < 1e-13


def test_own_route_tensor_T2_equals_library():
    """T^(2) by the own inverse DFT equals the library route (Eq. Tensor2)."""
    L, n, eps = (3.0, 4.0, 2.5), (6, 8, 4), 0.6
    own = dft.ifftn(fsa.fourier_W(L, n, eps)).real
    assert np.abs(own - fsa.tensor_T2(L, n, eps)).max() <= 1e-14 * np.abs(own).max()


def test_table2_iso_case1_own_fft():
    """Table 2, 3-D double, isotropic Case I at h = 1/2 (n = 32, printed
    2.5036E-06), every DFT of the scheme by the oracle's own transform."""
    d = W.paper_case1(L=8.0, sigma2=0.8, gamma3=1.0, h_over_gamma=0.5)
    assert d.n[0] == 32
    err = fsa.rel_error(fsa.solve(d.L, d.n, 1.0, d.rho(), fft="own"), cf.density_potential(d))
    assert err == pytest.approx(2.5036e-6, rel=5e-4)


# ---- planted mistakes in the own DFT must fail the pins above -------------------

def _dft_pins_pass():
    for n in (4, 6, 9, 12):
        rng = np.random.default_rng(n)
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        j = np.arange(n)
        want = np.array([np.sum(x * np.exp(-2j * np.pi * j * k / n)) for k in range(n)])
        if np.abs(dft.fft_axis(x, 0) - want).max() > 1e-12:
            return False
    d = W.paper_case1(L=8.0, sigma2=0.8, gamma3=1.0, h_over_gamma=0.5)
    err = fsa.rel_error(fsa.solve(d.L, d.n, 1.0, d.rho(), fft="own"), cf.density_potential(d))
    return abs(err - 2.5036e-6) <= 5e-4 * 2.5036e-6


_orig_fft_last = dft._fft_last


def _fft_twiddle_sign(a, inverse):
    """Twiddles of the combine step with the opposite sign."""
    n = a.shape[-1]
    if n == 1 or n % 2:
        return _orig_fft_last(a, inverse)
    m = n // 2
    E, O = _fft_twiddle_sign(a[..., 0::2], inverse), _fft_twiddle_sign(a[..., 1::2], inverse)
    w = np.exp((-1.0 if inverse else 1.0) * 2j * np.pi * np.arange(m) / n)
    return np.concatenate([E + w * O, E - w * O], axis=-1)


def _fft_swapped_halves(a, inverse):
    """The two output halves of each radix-2 step exchanged."""
    out = _orig_fft_last(a, inverse)
    n = a.shape[-1]
    if n % 2:
        return out
    return np.concatenate([out[..., n // 2:], out[..., :n // 2]], axis=-1)


def _fft_no_odd_term(a, inverse):
    """The odd subsequence dropped from the radix-2 combine."""
    n = a.shape[-1]
    if n == 1 or n % 2:
        return _orig_fft_last(a, inverse)
    E = _fft_no_odd_term(a[..., 0::2], inverse)
    return np.concatenate([E, E], axis=-1)


def _fft_radix3_index(a, inverse):
    """Radix 3 reading the subsequences with stride n/3 instead of 3."""
    n = a.shape[-1]
    if n % 3 or n % 2 == 0:
        return _orig_fft_last(a, inverse)
    m = n // 3
    b = np.concatenate([a[..., s * m:(s + 1) * m] for s in range(3)], axis=-1)
    b = b.reshape(a.shape[:-1] + (3, m)).swapaxes(-1, -2).reshape(a.shape)
    return _orig_fft_last(b, inverse)


def test_unmutated_dft_pins_pass():
    assert _dft_pins_pass()


@pytest.mark.parametrize("mutant", [_fft_twiddle_sign, _fft_swapped_halves, _fft_no_odd_term, _fft_radix3_index])
def test_dft_mutation_caught(monkeypatch, mutant):
    monkeypatch.setattr(dft, "_fft_last", mutant)
    assert not _dft_pins_pass()
