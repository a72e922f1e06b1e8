"""The radial Gauss-Kronrod route to W (Sec. 2.2, Eq. Fourier-Symmetric) on
the host: the 15-point Kronrod rule the library computes, and W(k) by the
radial integral against the closed forms of Table 1 / Example 4 and against
an independent adaptive quadrature (scipy's, in the oracle)."""
import numpy as np
import pytest

from oracle import fsa as oracle


@pytest.fixture(scope="module")
def capi():
    from paper_2504_19410_gb300 import capi as c
    try:
        c.lib()
    except RuntimeError:
        import __graft_entry__ as g
        g.build()
    return c


def test_kronrod15_is_the_kronrod_extension_of_gauss7(capi):
    x, wk, wg = capi.fsa_gauss_kronrod15()
    x, wk, wg = np.array(x), np.array(wk), np.array(wg)
    assert np.all(np.diff(x) > 0) and np.allclose(x, -x[::-1], atol=1e-16)
    # the Gauss part is numpy's 7-point Gauss-Legendre rule
    gx, gw = np.polynomial.legendre.leggauss(7)
    assert np.allclose(x[1::2], gx, rtol=0, atol=1e-15) and np.allclose(wg[1::2], gw, rtol=0, atol=1e-15)
    assert np.all(wg[0::2] == 0) and np.all(wk > 0)
    # Kronrod: exact through degree 22 = 3n + 1; Gauss: through 13, not 14
    for deg in range(23):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.dot(wk, x ** deg) - exact) < 1e-15, deg
    assert abs(np.dot(wg, x ** 13)) < 1e-15
    assert abs(np.dot(wg, x ** 14) - 2.0 / 15) > 1e-5


KERNELS = [("coulomb3d", 1.0, 0.0), ("biharmonic3d", 0.8, 0.0), ("poisson2d", 0.7, 0.0), ("coulomb2d", 1.0, 0.0),
           ("biharmonic2d", 0.9, 0.0), ("yukawa3d", 0.8, 0.5), ("yukawa2d", 0.6, 2.0)]


@pytest.mark.parametrize("name,eps,lam", KERNELS)
def test_radial_w_matches_the_closed_forms(capi, name, eps, lam):
    spec = (name, lam) if name.startswith("yukawa") else name
    W = oracle.kernel_fns(spec)[1]
    w0 = abs(float(W(0.0, eps)))
    for k in [0.0, 0.05, 0.9, 3.0, 11.0, 30.0, 60.0]:
        got, err = capi.fsa_radial_w(capi.KERNELS[name], eps, k, kernel_param=lam)
        assert abs(got - float(W(k, eps))) <= 1e-15 * w0, (k, got, float(W(k, eps)))
        assert err <= 1e-15 * w0


@pytest.mark.parametrize("name,eps,lam", KERNELS[:5])
def test_radial_w_matches_an_independent_quadrature(capi, name, eps, lam):
    """scipy's adaptive quadrature of the same integral (the oracle's pinned
    What_by_quadrature_kernel) at a few k."""
    for k in [0.5, 4.0]:
        got, _ = capi.fsa_radial_w(capi.KERNELS[name], eps, k)
        want = float(oracle.What_by_quadrature_kernel(k, eps, name))
        assert abs(got - want) <= 1e-12 * abs(want)
