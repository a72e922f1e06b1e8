"""ctypes binding of libfsaconv with the C-ABI's own names.

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  Pointers are plain integers (device or host addresses); streams are
integers holding a cudaStream_t (0 = legacy default stream).  A non-OK status
raises FsaError carrying the library's message.  If the shared library has not
been built this module raises on first use; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfsaconv.so")

FSA_OK, FSA_ERR_INVALID_ARG, FSA_ERR_UNSUPPORTED, FSA_ERR_EPS, FSA_ERR_OOM, FSA_ERR_CUDA, \
    FSA_ERR_NOT_GENERATED, FSA_ERR_BUSY, FSA_ERR_TIMEOUT, FSA_ERR_DEVICE_TIMEOUT, FSA_ERR_NOT_FOUND = range(11)
FSA_KERNEL_COULOMB3D = 0
FSA_KERNEL_BIHARMONIC3D = 1
FSA_KERNEL_POISSON2D = 2
FSA_KERNEL_COULOMB2D = 3
FSA_KERNEL_BIHARMONIC2D = 4
FSA_KERNEL_DDI3D = 5
FSA_KERNEL_YUKAWA3D = 6
FSA_KERNEL_YUKAWA2D = 7
KERNELS = {"coulomb3d": FSA_KERNEL_COULOMB3D, "biharmonic3d": FSA_KERNEL_BIHARMONIC3D,
           "poisson2d": FSA_KERNEL_POISSON2D, "coulomb2d": FSA_KERNEL_COULOMB2D,
           "biharmonic2d": FSA_KERNEL_BIHARMONIC2D, "ddi3d": FSA_KERNEL_DDI3D,
           "yukawa3d": FSA_KERNEL_YUKAWA3D, "yukawa2d": FSA_KERNEL_YUKAWA2D}
KERNEL_DIM = {FSA_KERNEL_COULOMB3D: 3, FSA_KERNEL_BIHARMONIC3D: 3, FSA_KERNEL_POISSON2D: 2,
              FSA_KERNEL_COULOMB2D: 2, FSA_KERNEL_BIHARMONIC2D: 2, FSA_KERNEL_DDI3D: 3,
              FSA_KERNEL_YUKAWA3D: 3, FSA_KERNEL_YUKAWA2D: 2}
FSA_DDI_GRID, FSA_DDI_KERNEL = 0, 1
DDI_DERIVATIVES = {"grid": FSA_DDI_GRID, "kernel": FSA_DDI_KERNEL}
FSA_F32, FSA_F64 = 0, 1
FSA_REQ_QUEUED, FSA_REQ_RUNNING, FSA_REQ_DONE, FSA_REQ_FAILED = range(4)


class FsaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


class PlanOpts(C.Structure):
    _fields_ = [("eps", C.c_double), ("eps_tol", C.c_double), ("device", C.c_int), ("kernel_param", C.c_double),
                ("l2_chunk_mb", C.c_int), ("w_quadrature", C.c_int)]


class PlanInfo(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("L", C.c_double * 3), ("h", C.c_double * 3), ("eps", C.c_double),
                ("R0", C.c_double), ("eps_bound", C.c_double), ("dtype", C.c_int), ("device", C.c_int),
                ("generated", C.c_int), ("arithmetic", C.c_int), ("launches_per_apply", C.c_int),
                ("workspace_bytes", C.c_size_t),
                ("spectrum_bytes", C.c_size_t),
                ("spectrum", C.c_void_p), ("kernel", C.c_int), ("d", C.c_int), ("kernel_param", C.c_double),
                ("many_capacity", C.c_int),
                ("ddi_derivative", C.c_int),
                ("dipole_n", C.c_double * 3), ("dipole_m", C.c_double * 3),
                ("fused_fwd", C.c_int), ("fused_inv", C.c_int), ("w_quadrature", C.c_int), ("w_panels", C.c_int),
                ("pipe", C.c_int)]


class ServeOpts(C.Structure):
    _fields_ = [("max_inflight", C.c_int), ("streams", C.c_int), ("hbm_fraction", C.c_double),
                ("hbm_budget_bytes", C.c_size_t), ("plan_cache_max", C.c_int), ("queue_max", C.c_int),
                ("device", C.c_int), ("policy", C.c_int)]


class Request(C.Structure):
    _fields_ = [("kernel", C.c_int), ("d", C.c_int), ("L", C.c_double * 3), ("n", C.c_int * 3),
                ("dtype", C.c_int), ("eps", C.c_double), ("rho", C.c_void_p), ("phi", C.c_void_p),
                ("kernel_param", C.c_double)]


class ReqTimes(C.Structure):
    _fields_ = [("submit_s", C.c_double), ("admit_s", C.c_double), ("done_s", C.c_double),
                ("plan_hit", C.c_int), ("status", C.c_int)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("plan_hits", C.c_uint64), ("plan_misses", C.c_uint64), ("device_bytes_held", C.c_size_t),
                ("inflight", C.c_int), ("queued", C.c_int)]


_VP = C.c_void_p
_PROTOS = {
    "fsa_plan_create": (C.c_int, [C.POINTER(_VP), C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                  C.c_int, C.POINTER(PlanOpts)]),
    "fsa_plan_create_ddi3d": (C.c_int, [C.POINTER(_VP), C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_int,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, C.POINTER(PlanOpts)]),
    "fsa_tensor_generate": (C.c_int, [_VP, _VP]),
    "fsa_apply": (C.c_int, [_VP, _VP, _VP, _VP]),
    "fsa_apply_host": (C.c_int, [_VP, _VP, _VP, _VP]),
    "fsa_apply_noalloc": (C.c_int, [_VP, _VP, _VP, _VP]),
    "fsa_apply_batched": (C.c_int, [C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP), C.c_int, _VP]),
    "fsa_apply_batched_launches": (C.c_int, [C.POINTER(_VP), C.c_int, C.POINTER(C.c_int)]),
    "fsa_batched_mode_set": (C.c_int, [C.c_int]),
    "fsa_plan_reserve": (C.c_int, [_VP, C.c_int]),
    "fsa_apply_many": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(_VP), C.c_int, _VP]),
    "fsa_plan_info_get": (C.c_int, [_VP, C.POINTER(PlanInfo)]),
    "fsa_plan_destroy": (C.c_int, [_VP]),
    "fsa_plan_spectrum_copy": (C.c_int, [_VP, _VP, C.c_size_t, _VP]),
    "fsa_appendix_b_bound": (C.c_double, [C.c_double, C.c_double]),
    "fsa_appendix_b_bound_kernel": (C.c_double, [C.c_int, C.c_double, C.c_double]),
    "fsa_appendix_b_bound_kernel_param": (C.c_double, [C.c_int, C.c_double, C.c_double, C.c_double]),
    "fsa_status_string": (C.c_char_p, [C.c_int]),
    "fsa_last_error": (C.c_char_p, []),
    "fsa_autotune_set": (C.c_int, [C.c_int]),
    "fsa_fused_configs": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]),
    "fsa_fused_select": (C.c_int, [C.c_int, C.c_int, C.c_int]),
    "fsa_pipe_select": (C.c_int, [C.c_int, C.c_int]),
    "fsa_apply_graphs_set": (C.c_int, [C.c_int]),
    "fsa_device_fault": (C.c_int, [C.c_int, C.POINTER(C.c_uint), C.c_int]),
    "fsa_wait_selftest": (C.c_int, [C.c_int, C.POINTER(C.c_uint)]),
    "fsa_measure_alu_peak": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_float)]),
    "fsa_radial_w": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                               C.POINTER(C.c_double)]),
    "fsa_gauss_kronrod15": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "fsa_profiler_create": (C.c_int, [C.POINTER(_VP), C.c_int]),
    "fsa_apply_profiled": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "fsa_profiler_read": (C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "fsa_profiler_destroy": (C.c_int, [_VP]),
    "fsa_serve_create": (C.c_int, [C.POINTER(_VP), C.POINTER(ServeOpts)]),
    "fsa_serve_submit": (C.c_int, [_VP, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "fsa_serve_poll": (C.c_int, [_VP, C.c_uint64, C.c_double, C.POINTER(C.c_int), C.POINTER(ReqTimes)]),
    "fsa_serve_stats_get": (C.c_int, [_VP, C.POINTER(ServeStats)]),
    "fsa_serve_destroy": (C.c_int, [_VP]),
}

_lib = None


def lib():
    """Load libfsaconv.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfsaconv is not built ({LIB_PATH} missing): run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        handle = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _status_name(s):
    try:
        return lib().fsa_status_string(s).decode()
    except Exception:  # library not loadable
        return f"status {s}"


def check(status):
    if status != FSA_OK:
        raise FsaError(status, lib().fsa_last_error().decode())
    return status


def _ptr(x):
    """Accept an int address, None, or an object with data_ptr() (a torch tensor)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


# ---- the C-ABI calls, same names ------------------------------------------------

def fsa_plan_create(kernel, d, L, n, dtype, eps=0.0, eps_tol=0.0, device=-1, l2_chunk_mb=0, kernel_param=0.0,
                    w_quadrature=0):
    h = _VP()
    o = PlanOpts(eps=float(eps), eps_tol=float(eps_tol), device=int(device), kernel_param=float(kernel_param),
                 l2_chunk_mb=int(l2_chunk_mb), w_quadrature=int(w_quadrature))
    check(lib().fsa_plan_create(C.byref(h), int(kernel), int(d), (C.c_double * 3)(*[float(x) for x in L]),
                                (C.c_int * 3)(*[int(x) for x in n]), int(dtype), C.byref(o)))
    return h.value


def fsa_plan_create_ddi3d(L, n, dtype, dipole_n, dipole_m, derivative, eps=0.0, eps_tol=0.0, device=-1):
    h = _VP()
    o = PlanOpts(eps=float(eps), eps_tol=float(eps_tol), device=int(device), kernel_param=0.0, l2_chunk_mb=0)
    d3 = lambda v: (C.c_double * 3)(*[float(x) for x in v])
    check(lib().fsa_plan_create_ddi3d(C.byref(h), d3(L), (C.c_int * 3)(*[int(x) for x in n]), int(dtype),
                                      d3(dipole_n), d3(dipole_m), int(derivative), C.byref(o)))
    return h.value


def fsa_tensor_generate(plan, stream=None):
    return check(lib().fsa_tensor_generate(plan, _stream(stream)))


def fsa_apply(plan, rho, phi, stream=None):
    return check(lib().fsa_apply(plan, _ptr(rho), _ptr(phi), _stream(stream)))


def fsa_apply_noalloc(plan, rho, phi, stream=None):
    return check(lib().fsa_apply_noalloc(plan, _ptr(rho), _ptr(phi), _stream(stream)))


def fsa_apply_host(plan, rho_host, phi_host, stream=None):
    return check(lib().fsa_apply_host(plan, _ptr(rho_host), _ptr(phi_host), _stream(stream)))


def fsa_apply_batched(plans, rhos, phis, stream=None):
    k = len(plans)
    P = (_VP * k)(*plans)
    R = (_VP * k)(*[_ptr(r) for r in rhos])
    F = (_VP * k)(*[_ptr(f) for f in phis])
    return check(lib().fsa_apply_batched(P, R, F, k, _stream(stream)))


def fsa_batched_mode_set(mode):
    """0 auto (time 1 and 2 on a batch's first call), 1 mixed one launch per pass,
    2 shape groups only, 3 mixed pipelined in two halves."""
    return check(lib().fsa_batched_mode_set(int(mode)))


def fsa_apply_batched_launches(plans):
    """Kernel launches one fsa_apply_batched call over these plans makes."""
    k = len(plans)
    P = (_VP * k)(*plans)
    n = C.c_int()
    check(lib().fsa_apply_batched_launches(P, k, C.byref(n)))
    return n.value


def fsa_plan_reserve(plan, count):
    return check(lib().fsa_plan_reserve(plan, int(count)))


def fsa_apply_many(plan, rhos, phis, stream=None):
    k = len(rhos)
    R = (_VP * k)(*[_ptr(r) for r in rhos])
    F = (_VP * k)(*[_ptr(f) for f in phis])
    return check(lib().fsa_apply_many(plan, R, F, k, _stream(stream)))


def fsa_plan_info_get(plan):
    info = PlanInfo()
    check(lib().fsa_plan_info_get(plan, C.byref(info)))
    return info


def fsa_plan_spectrum_copy(plan, dst, nbytes, stream=None):
    return check(lib().fsa_plan_spectrum_copy(plan, _ptr(dst), int(nbytes), _stream(stream)))


def fsa_plan_destroy(plan):
    return check(lib().fsa_plan_destroy(plan))


def fsa_appendix_b_bound(R0, eps):
    return lib().fsa_appendix_b_bound(float(R0), float(eps))


def fsa_appendix_b_bound_kernel(kernel, R0, eps):
    return lib().fsa_appendix_b_bound_kernel(int(kernel), float(R0), float(eps))


def fsa_appendix_b_bound_kernel_param(kernel, param, R0, eps):
    return lib().fsa_appendix_b_bound_kernel_param(int(kernel), float(param), float(R0), float(eps))


def fsa_status_string(s):
    return lib().fsa_status_string(int(s)).decode()


def fsa_last_error():
    return lib().fsa_last_error().decode()


def fsa_autotune_set(mode):
    return check(lib().fsa_autotune_set(int(mode)))


def fsa_fused_configs(M):
    """[(CTAs per cluster, threads per CTA), ...] of the fused outer pass
    pairs for transform length M (empty: none)."""
    cs = (C.c_int * 4)()
    nt = (C.c_int * 4)()
    k = lib().fsa_fused_configs(int(M), cs, nt, 4)
    return [(cs[i], nt[i]) for i in range(min(k, 4))]


def fsa_fused_select(M, direction, c):
    """Pin the outer pair for length M: direction 0 forward, 1 inverse, 2
    both; c = 0 separate passes, c >= 1 fused configuration c - 1, -1 tuner."""
    return check(lib().fsa_fused_select(int(M), int(direction), int(c)))


def fsa_apply_graphs_set(enable):
    """1 (default): repeated fsa_apply / fsa_apply_host calls with the same
    plan and buffers replay a captured CUDA graph; 0: direct launches."""
    return check(lib().fsa_apply_graphs_set(int(enable)))


def fsa_pipe_select(M, c):
    """Pin the middle passes for FP32 transform length M: c = 1 the pipelined
    kernel, 0 the separate passes, -1 tuner."""
    return check(lib().fsa_pipe_select(int(M), int(c)))


def fsa_device_fault(device=-1, clear=False):
    """The device's wait-timeout word (0 = no bounded device wait gave up)."""
    code = C.c_uint(0)
    check(lib().fsa_device_fault(int(device), C.byref(code), 1 if clear else 0))
    return code.value


def fsa_radial_w(kernel, eps, k, kernel_param=0.0):
    """(W(k), error estimate) by the radial Gauss-Kronrod quadrature (host)."""
    w, e = C.c_double(), C.c_double()
    check(lib().fsa_radial_w(int(kernel), float(kernel_param), float(eps), float(k), C.byref(w), C.byref(e)))
    return w.value, e.value


def fsa_gauss_kronrod15():
    """(nodes, Kronrod weights, Gauss weights) of the 15-point rule on [-1, 1]."""
    x, wk, wg = (C.c_double * 15)(), (C.c_double * 15)(), (C.c_double * 15)()
    check(lib().fsa_gauss_kronrod15(x, wk, wg))
    return list(x), list(wk), list(wg)


def fsa_measure_alu_peak(kind, device=-1):
    """(lane operations per second, ms of the timed launch); kind 0 = FP32 FMA,
    1 = FP64 FMA, 2 = paired FP32 FMA (fma.rn.f32x2; one FMA = one lane operation)."""
    rate, ms = C.c_double(), C.c_float()
    check(lib().fsa_measure_alu_peak(int(device), int(kind), C.byref(rate), C.byref(ms)))
    return rate.value, ms.value


def fsa_wait_selftest(device=-1):
    """Runs one bounded device wait that nothing completes; returns the fault
    word it left (1 = the wait gave up and was recorded)."""
    code = C.c_uint(0)
    check(lib().fsa_wait_selftest(int(device), C.byref(code)))
    return code.value


def fsa_profiler_create(max_steps):
    h = _VP()
    check(lib().fsa_profiler_create(C.byref(h), int(max_steps)))
    return h.value


def fsa_apply_profiled(plan, rho, phi, stream, prof):
    return check(lib().fsa_apply_profiled(plan, _ptr(rho), _ptr(phi), _stream(stream), prof))


def fsa_profiler_read(prof):
    """Returns (pass_ms[5], step_ms, steps), averages over the recorded steps."""
    p = (C.c_double * 5)()
    t = C.c_double()
    k = C.c_int()
    check(lib().fsa_profiler_read(prof, p, C.byref(t), C.byref(k)))
    return list(p), t.value, k.value


def fsa_profiler_destroy(prof):
    return check(lib().fsa_profiler_destroy(prof))


def fsa_serve_create(max_inflight=0, streams=0, hbm_fraction=0.0, hbm_budget_bytes=0, plan_cache_max=0,
                     queue_max=0, device=-1, policy=0):
    h = _VP()
    o = ServeOpts(max_inflight, streams, hbm_fraction, hbm_budget_bytes, plan_cache_max, queue_max, device,
                  int(policy))
    check(lib().fsa_serve_create(C.byref(h), C.byref(o)))
    return h.value


def fsa_serve_submit(server, L, n, dtype, rho, phi, eps=0.0, kernel=FSA_KERNEL_COULOMB3D, kernel_param=0.0):
    L3 = list(map(float, L)) + [1.0] * (3 - len(L))
    n3 = list(map(int, n)) + [1] * (3 - len(n))
    req = Request(kernel, len(n), (C.c_double * 3)(*L3), (C.c_int * 3)(*n3), int(dtype),
                  float(eps), _ptr(rho), _ptr(phi), float(kernel_param))
    t = C.c_uint64()
    check(lib().fsa_serve_submit(server, C.byref(req), C.byref(t)))
    return t.value


def fsa_serve_poll(server, ticket, timeout_s=0.0):
    """Returns (state, ReqTimes).  A wait that runs out (FSA_ERR_TIMEOUT) returns
    the current state (QUEUED or RUNNING); NOT_FOUND and other errors raise."""
    st = C.c_int()
    tm = ReqTimes()
    rc = lib().fsa_serve_poll(server, C.c_uint64(ticket), float(timeout_s), C.byref(st), C.byref(tm))
    if rc != FSA_ERR_TIMEOUT:
        check(rc)
    return st.value, tm


def fsa_serve_stats_get(server):
    s = ServeStats()
    check(lib().fsa_serve_stats_get(server, C.byref(s)))
    return s


def fsa_serve_destroy(server):
    return check(lib().fsa_serve_destroy(server))
