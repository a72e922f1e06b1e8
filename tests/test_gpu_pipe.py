"""The pipelined middle passes (FP32 grids with n1 = n2: row forward, middle
pass and row inverse as one kernel fed by a work dispenser) on the CUDA path.

Each transform length is pinned in turn (fsa_pipe_select) and compared with
the FP64 oracle on the same seeded inputs (max-norm relative error <= 2e-6,
the FP32 tolerance), and with the separate passes of the same process.  The
dispenser's edge cases are covered by the plane counts: K0 = n0 + 1 planes
per solve from 5 (the lag clamps to 2) to 257, one solve and several solves
per launch (fsa_apply_many, fsa_apply_batched), whose results must equal the
single solves bit for bit (the same kernels and arithmetic per solve).
"""
import numpy as np
import pytest

import workloads as W
from oracle import fsa as oracle

pytestmark = pytest.mark.gpu

TOL32 = 2e-6
LENGTHS = (128, 192, 256, 384, 512)


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2504_19410_gb300 as fsa
    return fsa


@pytest.fixture
def capi(lib):
    """Restores the default selection (tuner decides) after each test."""
    from paper_2504_19410_gb300 import capi as c
    c.fsa_device_fault(clear=True)
    yield c
    for M in LENGTHS:
        c.fsa_pipe_select(M, -1)
    c.fsa_autotune_set(1)
    import torch
    torch.cuda.synchronize()


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def solve(lib, L, n, eps, rho):
    import torch
    plan = lib.Plan(L, n, "f32", eps=eps)
    out = plan.apply(to_dev(rho))
    torch.cuda.synchronize()
    info = plan.info
    res = out.double().cpu().numpy()
    plan.close()
    return res, info


@pytest.mark.parametrize("n0", [4, 12, 24])
@pytest.mark.parametrize("M", LENGTHS)
def test_pipe_matches_oracle(lib, capi, M, n0):
    n = (n0, M // 2, M // 2)
    capi.fsa_autotune_set(0)
    rng = np.random.default_rng(M + 11 * n0)
    L = (1.0 + n0 / 16, 2.5, 3.0)
    rho = rng.standard_normal(n)
    want = oracle.solve(L, n, 0.5, rho)
    capi.fsa_pipe_select(M, 1)
    got, info = solve(lib, L, n, 0.5, rho)
    assert info.pipe == 1 and info.launches_per_apply == 3
    assert capi.fsa_device_fault(clear=True) == 0
    capi.fsa_pipe_select(M, 0)
    sep, info0 = solve(lib, L, n, 0.5, rho)
    assert info0.pipe == 0
    e_pipe = oracle.rel_error(got, want)
    e_sep = oracle.rel_error(sep, want)
    e_pair = oracle.rel_error(got, sep)
    print(f"\nM={M} n={n}: pipelined {e_pipe:.3e}, separate {e_sep:.3e}, pipelined vs separate {e_pair:.3e}")
    assert e_pipe <= TOL32
    assert e_pair <= 1e-6


def test_pipe_256_every_output_and_repeatable(lib, capi):
    """The 256^3 workload through the pipelined kernel: every output against
    the oracle's FFT route and against the separate passes, and two launches
    in a row equal (the counters are cleared per launch)."""
    import torch
    d = W.gaussian_sum(seed=2504)
    rho = d.rho()
    capi.fsa_autotune_set(1)
    capi.fsa_pipe_select(512, 1)
    plan = lib.Plan(d.L, d.n, "f32", eps=d.eps)
    assert plan.info.pipe == 1
    x = to_dev(rho)
    a = plan.apply(x)
    b = plan.apply(x)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert capi.fsa_device_fault(clear=True) == 0
    got = a.double().cpu().numpy()
    plan.close()
    capi.fsa_pipe_select(512, 0)
    sep, _ = solve(lib, d.L, d.n, d.eps, rho)
    e_pair = oracle.rel_error(got, sep)
    want = oracle.apply_spectrum(oracle.spectrum(oracle.tensor_T(d.L, d.n, d.eps)), rho)
    e_all = oracle.rel_error(got, want)
    print(f"\n256^3 pipelined: every output vs oracle {e_all:.3e}, vs separate passes {e_pair:.3e}")
    assert e_pair <= 1e-6
    assert e_all <= TOL32


def test_pipe_many_and_batched_equal_single(lib, capi):
    """Several solves per launch share one dispenser (planes of all jobs in one
    order): each result equals its single solve bit for bit."""
    import torch
    from paper_2504_19410_gb300 import capi as c
    n = (12, 64, 64)
    L = (2.0, 2.5, 3.0)
    capi.fsa_autotune_set(0)
    capi.fsa_pipe_select(128, 1)
    rng = np.random.default_rng(3)
    rhos = [to_dev(rng.standard_normal(n)) for _ in range(3)]
    plan = lib.Plan(L, n, "f32", eps=0.5)
    assert plan.info.pipe == 1
    single = [plan.apply(r) for r in rhos]
    plan.reserve(3)
    many = [torch.empty_like(r) for r in rhos]
    plan.apply_many(rhos, many)
    plans = [lib.Plan(L, n, "f32", eps=0.5) for _ in range(3)]
    outs = [torch.empty_like(r) for r in rhos]
    c.fsa_batched_mode_set(2)  # shape groups: the group's passes, here the pipelined kernel
    try:
        lib.apply_batched(plans, rhos, outs)
    finally:
        c.fsa_batched_mode_set(0)
    torch.cuda.synchronize()
    assert c.fsa_device_fault(clear=True) == 0
    for k in range(3):
        assert torch.equal(many[k], single[k])
        assert torch.equal(outs[k], single[k])
    want = oracle.solve(L, n, 0.5, rhos[1].double().cpu().numpy())
    assert oracle.rel_error(single[1].double().cpu().numpy(), want) <= TOL32
    for p in plans:
        p.close()
    plan.close()
