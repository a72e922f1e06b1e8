"""The bounded device-side wait of the bulk-copy row passes, exercised on the
GPU without a fault: a kernel waits on an mbarrier that nothing completes, its
wait gives up after about 1 ms, the timeout lands in the device's fault word,
and the context stays usable (a solve afterwards still matches the oracle)."""
import numpy as np
import pytest

import oracle.fsa as oracle


@pytest.mark.gpu
def test_wait_gives_up_and_reports():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2504_19410_gb300 as fsa
    from paper_2504_19410_gb300 import capi

    assert capi.fsa_wait_selftest() == 1  # bit 0: an mbarrier wait timed out
    assert capi.fsa_device_fault() == 0   # the self-test cleared the word again
    # the context is intact: a solve through the bulk-copy row passes still
    # matches the oracle and leaves no fault behind
    capi.fsa_autotune_set(5)
    try:
        n, L, eps = (16, 12, 8), (4.0, 3.0, 2.5), 0.8
        rho = np.random.default_rng(11).standard_normal(n)
        plan = fsa.Plan(L, n, "f32", eps=eps)
        out = plan.apply(torch.from_numpy(rho.astype(np.float32)).cuda())
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        plan.close()
    finally:
        capi.fsa_autotune_set(1)
    assert oracle.rel_error(got, oracle.solve(L, n, eps, rho)) <= 2e-6
    torch.cuda.synchronize()
    assert capi.fsa_device_fault() == 0
