"""Plans whose W comes from the radial Gauss-Kronrod quadrature
(fsa_plan_opts.w_quadrature = 1; Sec. 2.2, Eq. Fourier-Symmetric), on the GPU:
the stored spectrum and the solves against the oracle (whose W is the closed
form of Table 1 / Example 4) and against the closed-form plan."""
import numpy as np
import pytest

from oracle import fsa as oracle

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}
CASES = [("coulomb3d", (12, 16, 24), (2.0, 2.5, 3.0), 0.0), ("biharmonic3d", (16, 8, 12), (2.5, 2.0, 3.0), 0.0),
         ("yukawa3d", (8, 12, 16), (2.0, 3.0, 2.5), 0.5), ("poisson2d", (24, 16), (3.0, 2.0), 0.0),
         ("coulomb2d", (16, 32), (2.0, 3.0), 0.0), ("biharmonic2d", (12, 24), (3.0, 2.5), 0.0),
         ("yukawa2d", (16, 12), (2.0, 2.0), 2.0)]


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2504_19410_gb300 as fsa
    return fsa


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("name,n,L,lam", CASES)
def test_quadrature_plan_matches_oracle(lib, name, n, L, lam, dt):
    import torch
    eps = min(1.0, 2 * min(L) / 6)
    spec = (name, lam) if name.startswith("yukawa") else name
    plan = lib.Plan(L, n, dt, eps=eps, kernel=name, kernel_param=lam, w_quadrature=1)
    closed = lib.Plan(L, n, dt, eps=eps, kernel=name, kernel_param=lam)
    try:
        info = plan.info
        assert info.w_quadrature == 1 and info.w_panels > 0 and closed.info.w_quadrature == 0
        T = oracle.tensor_T(L, n, eps, kernel=spec)
        want_S = oracle.spectrum_octant(T, n)
        got_S = plan.spectrum().double().cpu().numpy().reshape(want_S.shape)
        assert oracle.rel_error(got_S, want_S) <= (1e-13 if dt == "f64" else 2e-7)
        cl_S = closed.spectrum().double().cpu().numpy().reshape(want_S.shape)
        assert oracle.rel_error(got_S, cl_S) <= (1e-13 if dt == "f64" else 2e-7)
        rho = np.random.default_rng(sum(n)).standard_normal(n)
        x = torch.from_numpy(rho.astype(np.float64 if dt == "f64" else np.float32)).cuda()
        got = plan.apply(x).double().cpu().numpy()
        torch.cuda.synchronize()
        err = oracle.rel_error(got, oracle.apply_fft(T, rho))
        assert err <= TOL[dt], err
    finally:
        plan.close()
        closed.close()


def test_quadrature_plan_at_the_headline_size(lib):
    """256^3 on [-16,16]^3, eps = 1, FP64: the quadrature spectrum equals the
    closed-form one (Table 1's 3-D Coulomb W) to FP64 round-off."""
    import torch
    L, n = (16.0, 16.0, 16.0), (256, 256, 256)
    q = lib.Plan(L, n, "f64", eps=1.0, w_quadrature=1)
    c = lib.Plan(L, n, "f64", eps=1.0)
    try:
        a, b = q.spectrum(), c.spectrum()
        torch.cuda.synchronize()
        err = float((a - b).abs().max() / b.abs().max())
        print(f"256^3 quadrature W: {q.info.w_panels} Chebyshev panels, spectrum vs closed form {err:.2e}")
        assert err <= 1e-14
    finally:
        q.close()
        c.close()
