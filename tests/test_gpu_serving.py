"""The serving loop and the batched launcher on the GPU.

Serving is continuous batching: requests submitted while others run are
admitted as slots and HBM free up and overlap on the device.  Each result
must equal the same request solved alone (fsa_apply on its own plan) bit for
bit: every request runs the same kernels on its own workspace, and nothing
is reduced across requests.
"""
import numpy as np
import pytest

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


def make_requests(seed, count, sizes=(16, 24, 32, 48, 64)):
    import torch
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(rng.choice(sizes))
        nn = (n, n, int(rng.choice(sizes)))
        dt = "f64" if rng.uniform() < 0.3 else "f32"
        L = (4.0, 4.0, 2.0 + nn[2] / 16)
        tdt = torch.float64 if dt == "f64" else torch.float32
        rho = torch.from_numpy(rng.standard_normal(nn)).to(tdt).cuda()
        reqs.append((L, nn, dt, rho))
    return reqs


def alone(lib, L, n, dt, rho):
    import torch
    p = lib.Plan(L, n, dt, eps=0.0)
    out = p.apply(rho)
    torch.cuda.synchronize()
    p.close()
    return out


def test_served_results_equal_solved_alone(lib):
    import torch
    reqs = make_requests(1, 40)
    want = [alone(lib, *r) for r in reqs]
    srv = lib.Server(max_inflight=8, streams=4)
    outs = [torch.full_like(r[3], float("nan")) for r in reqs]
    tickets = []
    for k, (L, n, dt, rho) in enumerate(reqs):
        tickets.append(srv.submit(L, n, dt, rho, outs[k]))
        if k % 7 == 3:  # let some finish while more arrive
            srv.wait(tickets[k - 2])
    hits = 0
    for k, t in enumerate(tickets):
        try:
            tm = srv.wait(t)
            hits += tm.plan_hit
            assert tm.done_s >= tm.admit_s >= tm.submit_s
        except lib.FsaError as e:
            if "unknown ticket" not in str(e):  # already reported by the early wait
                raise
    torch.cuda.synchronize()
    for k in range(len(reqs)):
        assert torch.equal(outs[k], want[k]), k
    st = srv.stats()
    assert st.completed == len(reqs) and st.failed == 0 and st.inflight == 0
    assert st.plan_hits > 0
    srv.close()


def test_tight_hbm_budget_admits_in_turn(lib):
    """With room for about two workspaces the server still completes every
    request, admitting new ones only as earlier ones free their memory."""
    import torch
    reqs = make_requests(2, 12, sizes=(64,))
    want = [alone(lib, *r) for r in reqs]
    ws = 6 * 65 * 64 * 64 * 8
    srv = lib.Server(max_inflight=16, streams=4, hbm_budget_bytes=2 * ws + 3 * 65 ** 3 * 8)
    outs = [torch.empty_like(r[3]) for r in reqs]
    tickets = [srv.submit(L, n, dt, rho, outs[k]) for k, (L, n, dt, rho) in enumerate(reqs)]
    for t in tickets:
        srv.wait(t)
    torch.cuda.synchronize()
    for k in range(len(reqs)):
        assert torch.equal(outs[k], want[k]), k
    srv.close()


def test_serving_rejects_bad_requests_and_unknown_tickets(lib):
    import torch
    from paper_2504_19410_gb300 import capi
    srv = lib.Server()
    x = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(capi.FsaError) as ei:
        srv.submit((1, 1, 1), (8, 8, 10), "f32", x, x)
    assert ei.value.status == capi.FSA_ERR_INVALID_ARG
    with pytest.raises(capi.FsaError) as ei:
        srv.poll(123456789)
    assert ei.value.status == capi.FSA_ERR_NOT_FOUND
    srv.close()


def test_batched_c4_mix_equals_single(lib):
    """The C4-style mix (cubic n from {64,...,256}, gamma in {1,4,8}) in one
    batched call.  Under the default (auto) schedule, whichever of the mixed
    path and the shape groups it keeps, each result matches its solve alone
    within FP32 round-off and the oracle within the FP32 tolerance, and a
    repeated call (graph replay) gives the same bits.  Forced schedules: the
    mixed path in one launch per pass and pipelined give the same bits; the
    shape groups give fsa_apply's bits."""
    import torch
    import workloads as W
    from oracle import fsa as oracle
    dens = W.batch_requests(seed=2504, count=10, sizes=(64, 96, 128))
    plans, rhos, singles = [], [], []
    for d in dens:
        p = lib.Plan(d.L, d.n, "f32", eps=d.eps)
        r = torch.from_numpy(d.rho()).float().cuda()
        singles.append(p.apply(r).clone())
        plans.append(p)
        rhos.append(r)
    outs = [torch.full_like(r, float("nan")) for r in rhos]
    lib.apply_batched(plans, rhos, outs)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(float("nan"))
    lib.apply_batched(plans, rhos, outs)
    torch.cuda.synchronize()
    for d, s, o, f in zip(dens, singles, outs, first):
        assert torch.equal(o, f)
        a, b = o.double().cpu().numpy(), s.double().cpu().numpy()
        assert oracle.rel_error(a, b) <= 1e-6
        assert oracle.rel_error(a, oracle.solve(d.L, d.n, d.eps, d.rho())) <= 2e-6
    # the other schedules: one mixed launch per pass gives the same bits as the
    # pipelined default; the per-shape groups give fsa_apply's bits
    from paper_2504_19410_gb300 import capi
    handles = [p.handle for p in plans]
    auto_launches = capi.fsa_apply_batched_launches(handles)
    try:
        capi.fsa_batched_mode_set(1)
        mixed = None
        for mode in (1, 3, 2):
            capi.fsa_batched_mode_set(mode)
            if mode == 1:
                assert capi.fsa_apply_batched_launches(handles) == 5
            if mode == 3:
                assert capi.fsa_apply_batched_launches(handles) == 6
            if mode == 2:
                grouped_launches = capi.fsa_apply_batched_launches(handles)
                assert grouped_launches > 6
            for o in outs:
                o.fill_(float("nan"))
            lib.apply_batched(plans, rhos, outs)
            torch.cuda.synchronize()
            if mode == 1:
                mixed = [o.clone() for o in outs]
            want = singles if mode == 2 else mixed
            for o, w in zip(outs, want):
                assert torch.equal(o, w), mode
    finally:
        capi.fsa_batched_mode_set(0)
    # the auto mode kept one of the two candidates: its results are that one's
    # bits and its launch count that one's
    kept_mixed = all(torch.equal(f, m) for f, m in zip(first, mixed))
    assert kept_mixed or all(torch.equal(f, s) for f, s in zip(first, singles))
    assert auto_launches == (5 if kept_mixed else grouped_launches)
    for p in plans:
        p.close()


def test_served_kernels_do_not_share_plans(lib):
    """Coulomb and biharmonic requests on the same grid, box and eps are
    cached as different plans; each result equals its kernel's plan alone."""
    import torch
    rng = np.random.default_rng(5)
    L, n = (3.0, 3.0, 2.5), (16, 24, 16)
    rho = torch.from_numpy(rng.standard_normal(n)).cuda()
    want = {}
    for k in ("coulomb3d", "biharmonic3d"):
        p = lib.Plan(L, n, "f64", eps=0.0, kernel=k)
        want[k] = p.apply(rho)
        torch.cuda.synchronize()
        p.close()
    srv = lib.Server(max_inflight=4, streams=2)
    outs, tickets = {}, {}
    for rep in range(2):
        for k in ("coulomb3d", "biharmonic3d"):
            outs[(k, rep)] = torch.full_like(rho, float("nan"))
            tickets[(k, rep)] = srv.submit(L, n, "f64", rho, outs[(k, rep)], kernel=k)
    for key, t in tickets.items():
        srv.wait(t)
    torch.cuda.synchronize()
    srv.close()
    for (k, rep), o in outs.items():
        assert torch.equal(o, want[k]), (k, rep)
    assert not torch.equal(want["coulomb3d"], want["biharmonic3d"])


def test_served_plane_requests_equal_solved_alone(lib):
    """Plane (d = 2) requests are served beside 3-D ones; each equals its plan
    solved alone."""
    import torch
    rng = np.random.default_rng(8)
    reqs = [("poisson2d", (4.0, 4.0), (32, 48), "f32"), ("coulomb3d", (3.0, 3.0, 3.0), (16, 16, 16), "f64"),
            ("biharmonic2d", (5.0, 3.0), (64, 32), "f64"), ("coulomb2d", (4.0, 4.0), (48, 48), "f32")]
    want, outs, tickets, rhos = [], [], [], []
    srv = lib.Server(max_inflight=4, streams=2)
    for kernel, L, n, dt in reqs:
        tdt = torch.float64 if dt == "f64" else torch.float32
        rho = torch.from_numpy(rng.standard_normal(n)).to(tdt).cuda()
        rhos.append(rho)
        p = lib.Plan(L, n, dt, eps=0.0, kernel=kernel)
        want.append(p.apply(rho))
        torch.cuda.synchronize()
        p.close()
        outs.append(torch.full_like(rho, float("nan")))
        tickets.append(srv.submit(L, n, dt, rho, outs[-1], kernel=kernel))
    for t in tickets:
        srv.wait(t)
    torch.cuda.synchronize()
    srv.close()
    from oracle import fsa as oracle
    for i, (o, w) in enumerate(zip(outs, want)):
        kernel, L, n, dt = reqs[i]
        ref = oracle.solve(L, n, min(1.0, 2 * min(L) / 6), rhos[i].double().cpu().numpy(), kernel=kernel)
        e_srv = oracle.rel_error(o.double().cpu().numpy(), ref)
        e_alone = oracle.rel_error(w.double().cpu().numpy(), ref)
        assert torch.equal(o, w), (reqs[i], e_srv, e_alone)
        assert e_srv <= (1e-12 if dt == "f64" else 2e-6), (reqs[i], e_srv)


@pytest.mark.parametrize("kernel,L,n,lam", [("yukawa3d", (3.0, 2.5, 3.5), (16, 24, 32), 0.5),
                                            ("yukawa2d", (3.0, 4.0), (48, 32), 2.0)])
def test_served_yukawa_request_with_lambda(lib, kernel, L, n, lam):
    """A Yukawa request carries its lam (kernel_param): the served result
    equals the plan solved alone with that lam and the oracle's solve for it
    (Example 4's screened kernels), in both tiers."""
    import torch
    from oracle import fsa as oracle
    rng = np.random.default_rng(21)
    srv = lib.Server(max_inflight=4, streams=2)
    try:
        for dt in ("f64", "f32"):
            tdt = torch.float64 if dt == "f64" else torch.float32
            rho = torch.from_numpy(rng.standard_normal(n)).to(tdt).cuda()
            p = lib.Plan(L, n, dt, eps=0.0, kernel=kernel, kernel_param=lam)
            eps = p.eps
            want = p.apply(rho)
            torch.cuda.synchronize()
            p.close()
            out = torch.full_like(rho, float("nan"))
            srv.wait(srv.submit(L, n, dt, rho, out, kernel=kernel, kernel_param=lam))
            torch.cuda.synchronize()
            assert torch.equal(out, want)
            ref = oracle.solve(L, n, eps, rho.double().cpu().numpy(), kernel=(kernel, lam))
            err = oracle.rel_error(out.double().cpu().numpy(), ref)
            assert err <= (1e-12 if dt == "f64" else 2e-6), (dt, err)
            # lam = 1 is a different plan: its result differs
            other = torch.full_like(rho, float("nan"))
            srv.wait(srv.submit(L, n, dt, rho, other, kernel=kernel, kernel_param=1.0))
            torch.cuda.synchronize()
            assert not torch.equal(other, out)
    finally:
        srv.close()


def test_server_charges_each_plan_its_real_bytes(lib):
    """Admission counts what a resident plan really holds: the spectrum octant
    in its dtype, a second (double-word) copy for FP64 plans, and no third
    axis for a plane.  After the requests finish the server holds exactly
    the plans, and the device's free memory fell by at least that."""
    import torch
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    srv = lib.Server(max_inflight=2, streams=2)
    reqs = [("coulomb3d", (3.0, 3.0, 3.0), (32, 48, 64), "f64"), ("poisson2d", (4.0, 4.0), (64, 96), "f32"),
            ("coulomb2d", (4.0, 3.0), (32, 48), "f64")]
    want = 0
    rng = np.random.default_rng(22)
    try:
        keep = []
        for kernel, L, n, dt in reqs:
            tdt = torch.float64 if dt == "f64" else torch.float32
            rho = torch.from_numpy(rng.standard_normal(n)).to(tdt).cuda()
            out = torch.empty_like(rho)
            keep += [rho, out]
            srv.wait(srv.submit(L, n, dt, rho, out, kernel=kernel))
            octant = int(np.prod([x + 1 for x in n]))
            want += octant * (16 if dt == "f64" else 4)
        torch.cuda.synchronize()
        st = srv.stats()
        assert st.completed == len(reqs) and st.inflight == 0
        assert st.device_bytes_held == want, (st.device_bytes_held, want)
        assert free0 - torch.cuda.mem_get_info()[0] >= want
    finally:
        srv.close()


@pytest.mark.parametrize("policy", [0, 1])
def test_bulk_lane_results_equal_solved_alone(lib, policy):
    """A request large enough for the bulk lane (256^3 FP64: its grids launch
    one CTA per tile on a low-priority stream under policy 0) served among
    small ones: every result equals its plan solved alone, bit for bit, under
    both scheduling policies."""
    import torch
    rng = np.random.default_rng(30 + policy)
    big = ((16.0, 16.0, 16.0), (256, 256, 256), "f64")
    smalls = [((4.0, 4.0, 3.0), (32, 32, 16), "f32"), ((4.0, 3.0, 4.0), (48, 24, 32), "f64"),
              ((3.0, 3.0, 3.0), (64, 64, 64), "f32")]
    reqs = [big] + smalls * 3
    rhos, wants = [], []
    for L, n, dt in reqs:  # solved alone first (the plans tune the kernels of their sizes)
        tdt = torch.float64 if dt == "f64" else torch.float32
        rhos.append(torch.from_numpy(rng.standard_normal(n)).to(tdt).cuda())
        p = lib.Plan(L, n, dt, eps=0.0)
        wants.append(p.apply(rhos[-1]))
        torch.cuda.synchronize()
        p.close()
    srv = lib.Server(max_inflight=8, streams=4, policy=policy)
    try:
        outs = [torch.full_like(r, float("nan")) for r in rhos]
        tickets = [srv.submit(L, n, dt, rho, out) for (L, n, dt), rho, out in zip(reqs, rhos, outs)]
        for t in tickets:
            srv.wait(t)
        torch.cuda.synchronize()
        for (L, n, dt), out, want in zip(reqs, outs, wants):
            assert torch.equal(out, want), (n, dt)
    finally:
        srv.close()
