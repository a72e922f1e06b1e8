"""The C-ABI library builds, loads and exports what include/*.h declares;
host-only logic (argument validation, the App. B bound) is checked without a
GPU.  No call here launches device work."""
import glob
import math
import os
import re

import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="session")
def capi():
    import __graft_entry__ as g
    g.build()
    from paper_2504_19410_gb300 import capi as c
    return c


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(fsa_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("fsa_plan_create", "fsa_tensor_generate", "fsa_apply", "fsa_apply_batched",
                 "fsa_serve_submit", "fsa_serve_poll", "fsa_plan_destroy", "fsa_status_string"):
        assert want in names


def test_library_exports_every_declared_symbol(capi):
    lib = capi.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_status_strings(capi):
    assert capi.fsa_status_string(capi.FSA_OK) == "FSA_OK"
    assert capi.fsa_status_string(capi.FSA_ERR_EPS) == "FSA_ERR_EPS"


def test_appendix_b_bound_matches_oracle(capi):
    from oracle import fsa
    for R0, c in [(24.0, 5.85), (24.0, 5.8), (16.0, 6.0), (4.0, 10.0), (2.0, 4.0)]:
        a = capi.fsa_appendix_b_bound(R0, R0 / c)
        b = fsa.appendix_b_bound(R0, R0 / c)
        assert a == pytest.approx(b, rel=1e-8)
    assert math.isnan(capi.fsa_appendix_b_bound(0.0, 1.0))


def test_appendix_b_bound_per_kernel_matches_oracle(capi):
    """The library's closed forms of the far-field integral per kernel against
    the oracle's quadrature of the same integral."""
    from oracle import fsa
    for name, k in (("coulomb3d", capi.FSA_KERNEL_COULOMB3D), ("biharmonic3d", capi.FSA_KERNEL_BIHARMONIC3D)):
        for R0, eps in [(24.0, 1.0), (24.0, 4.1), (16.0, 2.7), (4.0, 0.9), (2.0, 0.5), (8.0, 2.0)]:
            a = capi.fsa_appendix_b_bound_kernel(k, R0, eps)
            b = fsa.appendix_b_bound(R0, eps, kernel=name)
            assert a == pytest.approx(b, rel=1e-8, abs=1e-300), (name, R0, eps)
    for name, k in (("poisson2d", capi.FSA_KERNEL_POISSON2D), ("coulomb2d", capi.FSA_KERNEL_COULOMB2D),
                    ("biharmonic2d", capi.FSA_KERNEL_BIHARMONIC2D)):
        for R0, eps in [(24.0, 24.0 / 5.64), (24.0, 24.0 / 5.75), (16.0, 2.7), (4.0, 0.9), (2.0, 0.5), (8.0, 2.0)]:
            a = capi.fsa_appendix_b_bound_kernel(k, R0, eps)
            b = fsa.appendix_b_bound(R0, eps, kernel=name)
            assert a == pytest.approx(b, rel=1e-8, abs=1e-300), (name, R0, eps)
    assert math.isnan(capi.fsa_appendix_b_bound_kernel(9, 24.0, 1.0))
    assert math.isnan(capi.fsa_appendix_b_bound_kernel(capi.FSA_KERNEL_BIHARMONIC3D, 24.0, 0.0))


def test_plan_create_checks_the_biharmonic_bound(capi):
    # R0 = 16, eps = 5: (eps^4/(8 pi)) int_{3.2}^inf s^3 erfc(s) ds ~ 1e-4 > 1e-8
    with pytest.raises(capi.FsaError) as ei:
        capi.fsa_plan_create(capi.FSA_KERNEL_BIHARMONIC3D, 3, (8, 8, 8), (8, 8, 8), capi.FSA_F32, eps=5.0)
    assert ei.value.status == capi.FSA_ERR_EPS


@pytest.mark.parametrize("n,L,kw,status", [
    ((4, 4, 5), (1, 1, 1), {}, "FSA_ERR_INVALID_ARG"),        # odd n
    ((4, 4, 10), (1, 1, 1), {}, "FSA_ERR_INVALID_ARG"),       # 10 = 2 * 5 not 2^a 3^b
    ((4, 4, 1024), (1, 1, 1), {}, "FSA_ERR_INVALID_ARG"),     # too large
    ((2, 4, 4), (1, 1, 1), {}, "FSA_ERR_INVALID_ARG"),        # too small
    ((8, 8, 8), (1, 0, 1), {}, "FSA_ERR_INVALID_ARG"),        # L <= 0
    ((8, 8, 8), (1, 1, 1), {"eps": -1.0}, "FSA_ERR_INVALID_ARG"),
    ((8, 8, 8), (8, 8, 8), {"eps": 5.0}, "FSA_ERR_EPS"),      # R0/eps = 3.2: bound ~ 4e-5 > 1e-8
    ((8, 8, 8), (8, 8, 8), {"eps": 3.0, "eps_tol": 1e-16}, "FSA_ERR_EPS"),
])
def test_plan_create_rejects_before_touching_the_device(capi, n, L, kw, status):
    with pytest.raises(capi.FsaError) as ei:
        capi.fsa_plan_create(capi.FSA_KERNEL_COULOMB3D, 3, L, n, capi.FSA_F32, **kw)
    assert capi.fsa_status_string(ei.value.status) == status


def test_fp64_plans_default_to_the_16_digit_tolerance(capi):
    """App. B: eps_tol = 1e-16 for 16 digits.  eps = 3 on [-8,8]^3 (R0 = 16,
    c = 5.33) has a bound between 1e-16 and 1e-8: an FP32 plan takes it by
    default, an FP64 plan rejects it unless the caller loosens eps_tol."""
    b = capi.fsa_appendix_b_bound(16.0, 3.0)
    assert 1e-16 < b < 1e-8
    with pytest.raises(capi.FsaError) as ei:
        capi.fsa_plan_create(capi.FSA_KERNEL_COULOMB3D, 3, (8, 8, 8), (8, 8, 8), capi.FSA_F64, eps=3.0)
    assert ei.value.status == capi.FSA_ERR_EPS
    for dt, kw in ((capi.FSA_F32, {}), (capi.FSA_F64, {"eps_tol": 1e-8})):
        try:
            capi.fsa_plan_destroy(capi.fsa_plan_create(capi.FSA_KERNEL_COULOMB3D, 3, (8, 8, 8), (8, 8, 8), dt,
                                                       eps=3.0, **kw))
        except capi.FsaError as e:  # without a device, creation stops after validation
            assert e.status != capi.FSA_ERR_EPS


def test_plan_create_rejects_dimension_and_kernel(capi):
    with pytest.raises(capi.FsaError) as ei:
        capi.fsa_plan_create(capi.FSA_KERNEL_COULOMB3D, 2, (1, 1, 1), (8, 8, 8), capi.FSA_F32)
    assert ei.value.status == capi.FSA_ERR_INVALID_ARG
    with pytest.raises(capi.FsaError) as ei:
        capi.fsa_plan_create(9, 3, (1, 1, 1), (8, 8, 8), capi.FSA_F32)
    assert ei.value.status == capi.FSA_ERR_UNSUPPORTED


def test_supported_sizes_match_workloads(capi):
    import workloads
    for n in range(2, 600):
        ok = n in workloads.SUPPORTED_N
        try:
            h = capi.fsa_plan_create(capi.FSA_KERNEL_COULOMB3D, 3, (1, 1, 1), (n, 4, 4), capi.FSA_F32,
                                     eps=0.1, eps_tol=-1)
            capi.fsa_plan_destroy(h)  # only reached when a device is present
            accepted = True
        except capi.FsaError as e:
            accepted = e.status != capi.FSA_ERR_INVALID_ARG
        assert accepted == ok, n


def test_plan_create_checks_dimension_against_kernel(capi):
    for k, d in ((capi.FSA_KERNEL_POISSON2D, 3), (capi.FSA_KERNEL_COULOMB2D, 3), (capi.FSA_KERNEL_COULOMB3D, 2)):
        with pytest.raises(capi.FsaError) as ei:
            capi.fsa_plan_create(k, d, (1, 1, 1), (8, 8, 8), capi.FSA_F32)
        assert ei.value.status == capi.FSA_ERR_INVALID_ARG
    # plane kernels validate only their two axes
    with pytest.raises(capi.FsaError) as ei:
        capi.fsa_plan_create(capi.FSA_KERNEL_POISSON2D, 2, (1, 1), (8, 10), capi.FSA_F32)
    assert ei.value.status == capi.FSA_ERR_INVALID_ARG
    with pytest.raises(capi.FsaError) as ei:
        capi.fsa_plan_create(capi.FSA_KERNEL_COULOMB2D, 2, (8, 8), (8, 8), capi.FSA_F32, eps=5.0)
    assert ei.value.status == capi.FSA_ERR_EPS


def test_ddi_plan_create_rejects_before_touching_the_device(capi):
    """fsa_plan_create_ddi3d's argument checks (no device needed)."""
    good = dict(eps=0.5)
    cases = [
        ((1, 1, 1), (8, 4, 8), (0, 0, 1), (0, 0, 1), capi.FSA_DDI_GRID),       # grid reading needs n_j >= 8
        ((1, 1, 1), (8, 8, 8), (0, 0, float("nan")), (0, 0, 1), capi.FSA_DDI_KERNEL),
        ((1, 1, 1), (8, 8, 8), (0, 0, 1), (0, float("inf"), 1), capi.FSA_DDI_GRID),
        ((1, 1, 1), (8, 8, 8), (0, 0, 1), (0, 0, 1), 7),                         # unknown derivative
        ((1, 1, 1), (8, 8, 10), (0, 0, 1), (0, 0, 1), capi.FSA_DDI_KERNEL),    # unsupported n
    ]
    for L, n, dn, dm, der in cases:
        with pytest.raises(capi.FsaError) as ei:
            capi.fsa_plan_create_ddi3d(L, n, capi.FSA_F32, dn, dm, der, **good)
        assert ei.value.status == capi.FSA_ERR_INVALID_ARG, (n, dn, dm, der)
    with pytest.raises(capi.FsaError) as ei:  # Coulomb's App. B check applies
        capi.fsa_plan_create_ddi3d((8, 8, 8), (8, 8, 8), capi.FSA_F32, (0, 0, 1), (0, 0, 1), capi.FSA_DDI_GRID,
                                   eps=5.0)
    assert ei.value.status == capi.FSA_ERR_EPS
    with pytest.raises(capi.FsaError) as ei:  # DDI plans need their dipoles
        capi.fsa_plan_create(capi.FSA_KERNEL_DDI3D, 3, (1, 1, 1), (8, 8, 8), capi.FSA_F32)
    assert ei.value.status == capi.FSA_ERR_INVALID_ARG


def test_yukawa_bound_matches_oracle(capi):
    """The library's swapped-order quadrature of the Yukawa far-field integral
    against the oracle's adaptive quadrature of the same integral."""
    from oracle import fsa
    for name, k in (("yukawa3d", capi.FSA_KERNEL_YUKAWA3D), ("yukawa2d", capi.FSA_KERNEL_YUKAWA2D)):
        for R0, eps, lam in [(24.0, 4.0, 1.0), (16.0, 2.7, 0.5), (8.0, 1.0, 1.0), (4.0, 0.9, 3.0), (2.0, 0.5, 0.1)]:
            a = capi.fsa_appendix_b_bound_kernel_param(k, lam, R0, eps)
            b = fsa.appendix_b_bound(R0, eps, kernel=(name, lam))
            assert a == pytest.approx(b, rel=1e-9, abs=1e-300), (name, R0, eps, lam)
        assert math.isnan(capi.fsa_appendix_b_bound_kernel_param(k, 0.0, 8.0, 1.0))


def test_yukawa_plan_create_checks(capi):
    with pytest.raises(capi.FsaError) as ei:  # d mismatch
        capi.fsa_plan_create(capi.FSA_KERNEL_YUKAWA2D, 3, (1, 1, 1), (8, 8, 8), capi.FSA_F32)
    assert ei.value.status == capi.FSA_ERR_INVALID_ARG
    with pytest.raises(capi.FsaError) as ei:  # negative lam
        capi.fsa_plan_create(capi.FSA_KERNEL_YUKAWA3D, 3, (8, 8, 8), (8, 8, 8), capi.FSA_F32, eps=1.0, kernel_param=-1.0)
    assert ei.value.status == capi.FSA_ERR_INVALID_ARG
    with pytest.raises(capi.FsaError) as ei:  # App. B rejects a large eps (R0 = 4, eps = 2)
        capi.fsa_plan_create(capi.FSA_KERNEL_YUKAWA3D, 3, (2, 2, 2), (8, 8, 8), capi.FSA_F32, eps=2.0, kernel_param=0.5)
    assert ei.value.status == capi.FSA_ERR_EPS


def test_fused_configs_and_select_arguments(capi):
    """The fused outer pass pairs' cluster configurations are host-side
    registry data (no device needed); selection checks its arguments."""
    assert capi.fsa_fused_configs(512) == [(8, 128)]
    assert capi.fsa_fused_configs(384) == [(4, 128)]
    assert capi.fsa_fused_configs(256) == [(4, 256), (8, 128)]
    assert capi.fsa_fused_configs(128) == [(4, 64), (2, 64)]
    assert capi.fsa_fused_configs(64) == [(2, 64)]
    for M in (8, 32, 96, 192, 768, 1024, 2048, -2):
        assert capi.fsa_fused_configs(M) == []
    for args in ((192, 2, 1), (512, 3, 1), (512, -1, 0), (512, 2, 2), (512, 0, -2)):
        with pytest.raises(capi.FsaError) as ei:
            capi.fsa_fused_select(*args)
        assert ei.value.status == capi.FSA_ERR_INVALID_ARG
    for c in (-1, 0, 1):
        capi.fsa_fused_select(512, 2, c)
    capi.fsa_fused_select(512, 2, -1)


def test_pipe_select_arguments(capi):
    """The pipelined middle passes exist for FP32 lengths 128..512; selection
    checks its arguments (host-side registry data, no device needed)."""
    for args in ((64, 1), (96, 1), (1024, 1), (-2, 0), (512, 2), (512, -2)):
        with pytest.raises(capi.FsaError) as ei:
            capi.fsa_pipe_select(*args)
        assert ei.value.status == capi.FSA_ERR_INVALID_ARG
    for M in (128, 192, 256, 384, 512):
        for c in (1, 0, -1):
            capi.fsa_pipe_select(M, c)


def test_apply_graphs_set_arguments(capi):
    """The graph-replay switch takes 0 or 1 (host-side state, no device)."""
    for bad in (-1, 2, 7):
        with pytest.raises(capi.FsaError) as ei:
            capi.fsa_apply_graphs_set(bad)
        assert ei.value.status == capi.FSA_ERR_INVALID_ARG
    capi.fsa_apply_graphs_set(0)
    capi.fsa_apply_graphs_set(1)


def test_missing_library_fails_loudly(monkeypatch):
    """No fallback: with the shared library absent, the binding raises on its
    first call instead of computing anything another way."""
    from paper_2504_19410_gb300 import capi as c
    monkeypatch.setattr(c, "LIB_PATH", "/nonexistent/libfsaconv.so")
    monkeypatch.setattr(c, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        c.lib()
    with pytest.raises(RuntimeError, match="not built"):
        c.fsa_appendix_b_bound(16.0, 1.0)
