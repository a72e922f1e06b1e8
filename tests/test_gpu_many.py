"""fsa_apply_many: many densities through one plan in one launch sequence.

Every result must equal fsa_apply's on the same plan bit for bit (the same
kernels and arithmetic; the FP32 middle pass only changes the order in which
it visits tiles and reads each spectrum tile once for all densities), and
match the oracle within the usual tolerances.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fsa as oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2504_19410_gb300 as fsa
    return fsa


@pytest.fixture(params=["gen1", "gen2", "gen3", "gen4"])
def gen(request, lib):
    import torch
    from paper_2504_19410_gb300 import capi
    capi.fsa_device_fault(clear=True)
    capi.fsa_autotune_set({"gen1": 2, "gen2": 3, "gen3": 4, "gen4": 5}[request.param])
    yield request.param
    capi.fsa_autotune_set(1)
    torch.cuda.synchronize()
    assert capi.fsa_device_fault(clear=True) == 0


def densities(n, count, dt, seed):
    import torch
    rng = np.random.default_rng(seed)
    tdt = torch.float64 if dt == "f64" else torch.float32
    return [torch.from_numpy(rng.standard_normal(n)).to(tdt).cuda() for _ in range(count)]


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("n,count", [((16, 16, 16), 1), ((16, 24, 32), 3), ((32, 32, 32), 8), ((12, 8, 48), 5)])
def test_many_equals_single(lib, n, count, dt, gen):
    import torch
    L = (3.0, 2.5, 4.0)
    plan = lib.Plan(L, n, dt, eps=0.7)
    plan.reserve(count)
    assert plan.info.many_capacity == count
    rhos = densities(n, count, dt, seed=count)
    singles = [plan.apply(r).clone() for r in rhos]
    outs = plan.apply_many(rhos)
    torch.cuda.synchronize()
    for s, o in zip(singles, outs):
        assert torch.equal(s, o)
    want = oracle.solve(L, n, 0.7, rhos[-1].double().cpu().numpy())
    assert oracle.rel_error(outs[-1].double().cpu().numpy(), want) <= (1e-12 if dt == "f64" else 2e-6)
    plan.close()


def test_many_beyond_one_launch_table(lib):
    """70 densities: more than one job table (64 jobs per launch)."""
    import torch
    n = (8, 8, 8)
    plan = lib.Plan((2.0, 2.0, 2.0), n, "f32", eps=0.3)
    plan.reserve(70)
    rhos = densities(n, 70, "f32", seed=70)
    singles = [plan.apply(r).clone() for r in rhos]
    outs = plan.apply_many(rhos)
    torch.cuda.synchronize()
    assert all(torch.equal(s, o) for s, o in zip(singles, outs))
    plan.close()


@pytest.mark.parametrize("reading", ["grid", "kernel"])
@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_many_ddi_and_plane(lib, reading, dt):
    import torch
    n = (16, 8, 24)
    plan = lib.Plan((3.0, 2.0, 3.5), n, dt, eps=0.7, kernel="ddi3d", dipoles=W.ddi_dipoles(1),
                    ddi_derivative=reading)
    plan.reserve(4)
    rhos = densities(n, 4, dt, seed=4)
    singles = [plan.apply(r).clone() for r in rhos]
    outs = plan.apply_many(rhos)
    plane = lib.Plan((3.0, 2.0), (32, 24), dt, eps=0.7, kernel="poisson2d")
    plane.reserve(3)
    prhos = densities((32, 24), 3, dt, seed=3)
    psingles = [plane.apply(r).clone() for r in prhos]
    pouts = plane.apply_many(prhos)
    torch.cuda.synchronize()
    assert all(torch.equal(s, o) for s, o in zip(singles, outs))
    assert all(torch.equal(s, o) for s, o in zip(psingles, pouts))
    plan.close()
    plane.close()


def test_many_in_place_and_limits(lib):
    import torch
    from paper_2504_19410_gb300 import capi
    n = (16, 16, 16)
    plan = lib.Plan((2.0, 2.0, 2.0), n, "f32", eps=0.5)
    rhos = densities(n, 3, "f32", seed=5)
    singles = [plan.apply(r).clone() for r in rhos]
    with pytest.raises(capi.FsaError) as ei:  # capacity 1 until reserved
        plan.apply_many(rhos)
    assert ei.value.status == capi.FSA_ERR_INVALID_ARG
    with pytest.raises(capi.FsaError):
        capi.fsa_plan_reserve(plan.handle, 0)
    plan.reserve(2)
    plan.reserve(3)  # grows
    plan.reserve(1)  # never shrinks
    assert plan.info.many_capacity == 3
    plan.apply_many(rhos, rhos)  # in place
    torch.cuda.synchronize()
    assert all(torch.equal(s, o) for s, o in zip(singles, rhos))
    plan.close()
