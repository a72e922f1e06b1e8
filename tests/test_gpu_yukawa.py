"""Yukawa kernels (Example 4) on the CUDA path against the oracle.

Tensor generation differs from the other kernels (the 2-D U^eps and the 3-D
U^eps near r = 0 are Gauss-Legendre quadratures of the heat-kernel integral on
the device); the apply passes are the shared ones.  Tolerances as everywhere:
spectrum <= 1e-13 (FP64) / 2e-7 (FP32), solves <= 1e-12 / 2e-6.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as cf
from oracle import fsa as oracle

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2504_19410_gb300 as fsa
    return fsa


def to_dev(rho, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float64 if dt == "f64" else np.float32)).cuda()


CASES = [("yukawa3d", (8, 8, 8), (2.0, 2.0, 2.0), 1.0), ("yukawa3d", (12, 16, 24), (3.0, 3.0, 3.0), 0.3),
         ("yukawa3d", (16, 16, 16), (4.0, 4.0, 4.0), 3.0), ("yukawa2d", (16, 24), (3.0, 3.0), 1.0),
         ("yukawa2d", (64, 48), (6.0, 6.0), 0.5), ("yukawa2d", (8, 8), (2.0, 2.0), 2.0)]


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("kernel,n,L,lam", CASES)
def test_yukawa_spectrum_and_apply_match_oracle(lib, kernel, n, L, lam, dt):
    import torch
    eps = min(1.0, 2 * min(L) / 6)
    plan = lib.Plan(L, n, dt, eps=eps, kernel=kernel, kernel_param=lam)
    assert plan.info.kernel_param == lam
    T = oracle.tensor_T(L, n, eps, kernel=(kernel, lam))
    got = plan.spectrum().double().cpu().numpy().reshape([x + 1 for x in n])
    assert oracle.rel_error(got, oracle.spectrum_octant(T, n)) <= (1e-13 if dt == "f64" else 2e-7)
    rho = np.random.default_rng(sum(n)).standard_normal(n)
    out = plan.apply(to_dev(rho, dt)).double().cpu().numpy()
    torch.cuda.synchronize()
    assert oracle.rel_error(out, oracle.apply_fft(T, rho)) <= TOL[dt]
    plan.close()


@pytest.mark.parametrize("h", [0.5, 0.25])
def test_yukawa3d_accuracy_on_gpu(lib, h):
    """rho = exp(-|x|^2/1.2) on [-8,8]^3, eps = 1, lam = 1, FP64 tier: the
    oracle's spectral accuracy (4.2e-8 at h = 1/2, round-off at h = 1/4)."""
    L, s2 = 8.0, 1.2
    d = W.paper_case1(L=L, sigma2=s2, h_over_gamma=h)
    x = W.grid_axes(d.L, d.n)
    R = np.sqrt(x[0][:, None, None] ** 2 + x[1][None, :, None] ** 2 + x[2][None, None, :] ** 2)
    plan = lib.Plan(d.L, d.n, "f64", eps=1.0, kernel="yukawa3d", kernel_param=1.0)
    got = plan.apply(to_dev(d.rho(), "f64")).cpu().numpy()
    plan.close()
    err = oracle.rel_error(got, cf.yukawa3d_gaussian_r(s2, 1.0, R))
    print(f"yukawa3d h={h}: {err:.3e}")
    assert err < (5e-8 if h == 0.5 else 1e-13)


@pytest.mark.parametrize("h", [0.5, 0.25])
def test_yukawa2d_accuracy_on_gpu(lib, h):
    L, s2 = 8.0, 1.2
    n = int(round(2 * L / h))
    x = W.grid_axes((L, L), (n, n))
    R = np.sqrt(x[0][:, None] ** 2 + x[1][None, :] ** 2)
    plan = lib.Plan((L, L), (n, n), "f64", eps=1.0, kernel="yukawa2d", kernel_param=1.0)
    got = plan.apply(to_dev(np.exp(-R ** 2 / s2), "f64")).cpu().numpy()
    plan.close()
    err = oracle.rel_error(got, cf.yukawa2d_gaussian_r(s2, 1.0, R))
    print(f"yukawa2d h={h}: {err:.3e}")
    assert err < (3e-8 if h == 0.5 else 1e-13)


def test_yukawa_default_lambda_and_many(lib):
    """kernel_param 0 selects lam = 1; apply_many works on Yukawa plans."""
    import torch
    n, L = (16, 16, 16), (3.0, 3.0, 3.0)
    p0 = lib.Plan(L, n, "f32", eps=0.9, kernel="yukawa3d")
    p1 = lib.Plan(L, n, "f32", eps=0.9, kernel="yukawa3d", kernel_param=1.0)
    assert p0.info.kernel_param == 1.0
    assert torch.equal(p0.spectrum(), p1.spectrum())
    p0.reserve(3)
    rhos = [to_dev(np.random.default_rng(k).standard_normal(n), "f32") for k in range(3)]
    singles = [p0.apply(r).clone() for r in rhos]
    outs = p0.apply_many(rhos)
    torch.cuda.synchronize()
    assert all(torch.equal(s, o) for s, o in zip(singles, outs))
    p0.close()
    p1.close()
