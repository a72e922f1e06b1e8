"""fsa_apply_noalloc against fsa_apply, through the C-ABI.

fsa_apply_noalloc serves callers that cannot have device memory allocated on
their behalf (a framework whose caching allocator holds nearly all device
memory, or a host loop that must not block on cudaMalloc / cudaFree): it keeps
its scratch in a fixed 16 MiB static device array instead of the plan's
workspace.  Its results must match fsa_apply's within the tolerances the other
parity tests use, on consecutive calls that reuse the shared array.  This file
is collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module")
def capi():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2504_19410_gb300 import capi as c
    return c


def rel_error(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("dt,n", [("f32", (64, 64, 64)), ("f64", (64, 64, 64)), ("f64", (12, 48, 24)),
                                  ("f32", (6, 8, 96))])
def test_noalloc_matches_apply_on_two_calls(capi, dt, n):
    import torch
    tdt = torch.float32 if dt == "f32" else torch.float64
    L = (4.0, 3.0, 5.0)
    plan = capi.fsa_plan_create(capi.FSA_KERNEL_COULOMB3D, 3, L, n,
                                capi.FSA_F32 if dt == "f32" else capi.FSA_F64, eps=0.8)
    stream = torch.cuda.current_stream()
    capi.fsa_tensor_generate(plan, stream)
    rng = np.random.default_rng(11)
    try:
        for call in range(2):  # the second call finds the first call's data in the shared array
            rho = torch.from_numpy(rng.standard_normal(n)).to(tdt).cuda()
            ref = torch.empty_like(rho)
            out = torch.full_like(rho, float("nan"))
            capi.fsa_apply(plan, rho, ref, stream)
            capi.fsa_apply_noalloc(plan, rho, out, stream)
            torch.cuda.synchronize()
            a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
            assert np.isfinite(a).all()
            assert rel_error(a, b) <= TOL[dt], (call, rel_error(a, b))
    finally:
        capi.fsa_plan_destroy(plan)


def test_noalloc_rejects_grids_beyond_the_static_scratch(capi):
    import torch
    plan = capi.fsa_plan_create(capi.FSA_KERNEL_COULOMB3D, 3, (4.0, 4.0, 4.0), (96, 96, 96), capi.FSA_F64, eps=0.8)
    try:
        capi.fsa_tensor_generate(plan, torch.cuda.current_stream())
        x = torch.zeros((96, 96, 96), dtype=torch.float64, device="cuda")
        with pytest.raises(capi.FsaError) as ei:
            capi.fsa_apply_noalloc(plan, x, x, torch.cuda.current_stream())
        assert ei.value.status == capi.FSA_ERR_INVALID_ARG
        assert "static scratch" in str(ei.value)
    finally:
        torch.cuda.synchronize()
        capi.fsa_plan_destroy(plan)


@pytest.mark.parametrize("dt,derivative", [("f32", 0), ("f64", 0), ("f32", 1), ("f64", 1)])
def test_noalloc_matches_apply_for_ddi_plans(capi, dt, derivative):
    """3-D DDI plans (both readings) take the same static scratch: the grid
    reading's unpadded passes live inside the same X and Y regions."""
    import torch
    tdt = torch.float32 if dt == "f32" else torch.float64
    n = (32, 24, 48)
    plan = capi.fsa_plan_create_ddi3d((4.0, 3.0, 5.0), n, capi.FSA_F32 if dt == "f32" else capi.FSA_F64,
                                      (0.6, 0.0, 0.8), (0.0, 1.0, 0.0), derivative, eps=0.8)
    stream = torch.cuda.current_stream()
    capi.fsa_tensor_generate(plan, stream)
    rng = np.random.default_rng(13)
    try:
        for call in range(2):
            rho = torch.from_numpy(rng.standard_normal(n)).to(tdt).cuda()
            ref = torch.empty_like(rho)
            out = torch.full_like(rho, float("nan"))
            capi.fsa_apply(plan, rho, ref, stream)
            capi.fsa_apply_noalloc(plan, rho, out, stream)
            torch.cuda.synchronize()
            a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
            assert np.isfinite(a).all()
            assert rel_error(a, b) <= TOL[dt], (call, rel_error(a, b))
    finally:
        capi.fsa_plan_destroy(plan)


def test_noalloc_call_changes_no_free_memory(capi):
    """The static scratch is reserved when plans are made, so an apply through
    this entry point moves nothing in the device's free memory: not the first
    call after plan creation, and not later ones."""
    import torch
    n = (32, 32, 32)
    plan = capi.fsa_plan_create(capi.FSA_KERNEL_COULOMB3D, 3, (4.0, 4.0, 4.0), n, capi.FSA_F32, eps=0.8)
    stream = torch.cuda.current_stream()
    try:
        capi.fsa_tensor_generate(plan, stream)
        rho = torch.from_numpy(np.random.default_rng(3).standard_normal(n)).float().cuda()
        out = torch.empty_like(rho)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            capi.fsa_apply_noalloc(plan, rho, out, stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        capi.fsa_plan_destroy(plan)
