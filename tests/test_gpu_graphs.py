"""Repeated solves replayed from cached CUDA graphs (fsa_apply_graphs_set).

fsa_apply and fsa_apply_host capture the pass launches of a (plan, rho,
phi) triple on its second call and replay them afterwards.  A replay must
compute on the buffers' CURRENT contents and give the same bits as direct
launches; kernel selection changes must reach later calls; destroying a
plan must drop its graphs (a new plan, possibly at the same address, solves
correctly).
"""
import numpy as np
import pytest

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


@pytest.fixture
def capi(lib):
    from paper_2504_19410_gb300 import capi as c
    c.fsa_device_fault(clear=True)
    yield c
    c.fsa_apply_graphs_set(1)
    c.fsa_pipe_select(128, -1)
    c.fsa_autotune_set(1)


def dev(a, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32 if dt == "f32" else np.float64)).cuda()


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_replay_uses_current_contents_and_matches_direct(lib, capi, dt):
    import torch
    n, L = (12, 16, 24), (2.0, 2.5, 3.0)
    rng = np.random.default_rng(21)
    rhos = [rng.standard_normal(n) for _ in range(4)]
    plan = lib.Plan(L, n, dt, eps=0.5)
    x = dev(rhos[0], dt)
    y = torch.empty_like(x)
    capi.fsa_apply_graphs_set(0)
    direct = []
    for r in rhos:
        x.copy_(dev(r, dt))
        plan.apply(x, y)
        direct.append(y.clone())
    capi.fsa_apply_graphs_set(1)
    # call 1 direct, call 2 captured and replayed, calls 3-4 replayed: each on
    # new contents of the same buffers
    for k, r in enumerate(rhos):
        x.copy_(dev(r, dt))
        plan.apply(x, y)
        torch.cuda.synchronize()
        assert torch.equal(y, direct[k]), k
    want = oracle.solve(L, n, 0.5, rhos[3])
    assert oracle.rel_error(y.double().cpu().numpy(), want) <= (2e-6 if dt == "f32" else 1e-12)
    plan.close()


def test_selection_change_reaches_replayed_solves(lib, capi):
    """A graph keeps the kernels of its capture: fsa_pipe_select after two
    calls must still switch the next calls to the pipelined kernel (which
    computes the two-step passes' values; the separate passes of this
    process may be another generation, so the two agree to round-off)."""
    import torch
    n, L = (12, 64, 64), (2.0, 2.5, 3.0)
    capi.fsa_autotune_set(0)
    capi.fsa_pipe_select(128, 0)
    plan = lib.Plan(L, n, "f32", eps=0.5)
    x = dev(np.random.default_rng(3).standard_normal(n), "f32")
    y0 = torch.empty_like(x)
    for _ in range(3):
        plan.apply(x, y0)
    capi.fsa_pipe_select(128, 1)
    assert plan.info.pipe == 1
    y1 = torch.empty_like(x)
    for _ in range(3):
        plan.apply(x, y1)
    torch.cuda.synchronize()
    assert capi.fsa_device_fault(clear=True) == 0
    want = oracle.solve(L, n, 0.5, x.double().cpu().numpy())
    assert oracle.rel_error(y1.double().cpu().numpy(), want) <= 2e-6
    assert oracle.rel_error(y1.double().cpu().numpy(), y0.double().cpu().numpy()) <= 1e-6
    plan.close()


def test_selection_change_reaches_replayed_batches(lib, capi):
    """fsa_apply_batched's graphs are keyed on the kernel selection too: a
    batch captured with the separate passes is captured again once
    fsa_pipe_select pins the pipelined kernel, and each result then equals the
    single solve under the new selection bit for bit."""
    import torch
    n, L = (12, 64, 64), (2.0, 2.5, 3.0)
    capi.fsa_autotune_set(0)
    capi.fsa_pipe_select(128, 0)
    rng = np.random.default_rng(5)
    rhos = [dev(rng.standard_normal(n), "f32") for _ in range(2)]
    plans = [lib.Plan(L, n, "f32", eps=0.5) for _ in range(2)]
    solo = lib.Plan(L, n, "f32", eps=0.5)
    outs = [torch.empty_like(r) for r in rhos]
    capi.fsa_batched_mode_set(2)  # shape groups: the group's passes follow the selection
    try:
        for _ in range(2):
            lib.apply_batched(plans, rhos, outs)
        before = [solo.apply(r) for r in rhos]
        torch.cuda.synchronize()
        for k in range(2):
            assert torch.equal(outs[k], before[k]), k
        capi.fsa_pipe_select(128, 1)
        assert solo.info.pipe == 1
        for _ in range(2):
            lib.apply_batched(plans, rhos, outs)
        after = [solo.apply(r) for r in rhos]
        torch.cuda.synchronize()
    finally:
        capi.fsa_batched_mode_set(0)
    assert capi.fsa_device_fault(clear=True) == 0
    for k in range(2):
        assert torch.equal(outs[k], after[k]), k
    want = oracle.solve(L, n, 0.5, rhos[1].double().cpu().numpy())
    assert oracle.rel_error(outs[1].double().cpu().numpy(), want) <= 2e-6
    for p in plans + [solo]:
        p.close()


def test_destroyed_plan_drops_its_graphs(lib, capi):
    import torch
    rng = np.random.default_rng(8)
    for n in [(8, 12, 16), (16, 12, 8), (8, 12, 16)]:
        L = (2.0, 2.0, 2.0)
        plan = lib.Plan(L, n, "f64", eps=0.5)
        r = rng.standard_normal(n)
        x = dev(r, "f64")
        y = torch.empty_like(x)
        for _ in range(3):
            plan.apply(x, y)
        torch.cuda.synchronize()
        assert oracle.rel_error(y.cpu().numpy(), oracle.solve(L, n, 0.5, r)) <= 1e-12
        plan.close()


def test_host_entry_point_replays(lib, capi):
    """fsa_apply_host: copies in, passes (replayed from the second call on),
    copies out; each call computes on the host buffer's current contents."""
    import torch
    n, L = (12, 16, 24), (2.0, 2.5, 3.0)
    plan = lib.Plan(L, n, "f32", eps=0.5)
    rng = np.random.default_rng(4)
    host_in = torch.empty(n, dtype=torch.float32).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    for k in range(4):
        r = rng.standard_normal(n)
        host_in.copy_(torch.from_numpy(r.astype(np.float32)))
        plan.apply_host(host_in, host_out)
        torch.cuda.synchronize()
        direct = plan.apply(dev(r, "f32")).cpu()
        torch.cuda.synchronize()
        assert torch.equal(direct, host_out), k
    assert oracle.rel_error(host_out.double().numpy(), oracle.solve(L, n, 0.5, r)) <= 2e-6
    plan.close()


def test_apply_inside_a_callers_graph_capture(lib, capi):
    """A caller capturing its stream into its own CUDA graph gets the pass
    launches captured there (no capture or instantiation of the library's
    own inside it); replaying the caller's graph solves the current contents."""
    import torch
    n, L = (12, 16, 24), (2.0, 2.5, 3.0)
    plan = lib.Plan(L, n, "f32", eps=0.5)
    rng = np.random.default_rng(12)
    r0, r1 = rng.standard_normal(n), rng.standard_normal(n)
    x = dev(r0, "f32")
    y = torch.empty_like(x)
    for _ in range(2):  # the library's own graph of this triple exists by now
        plan.apply(x, y)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.apply(x, y, stream=s)
    x.copy_(dev(r1, "f32"))
    g.replay()
    torch.cuda.synchronize()
    assert capi.fsa_device_fault(clear=True) == 0
    want = oracle.solve(L, n, 0.5, r1)
    assert oracle.rel_error(y.double().cpu().numpy(), want) <= 2e-6
    plan.close()
