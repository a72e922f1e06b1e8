"""libfsaconv: the GB300 apply path of the FSA convolution solver (arXiv 2504.19410).

``capi`` exposes the C-ABI calls under their own names; ``Plan`` and
``Server`` wrap them for torch tensors.  Torch provides device memory and
streams only: every step of a solve runs in libfsaconv's CUDA kernels, and
there is no CPU path.  Build the library with ``__graft_entry__.build()``
(or ``python -m paper_2504_19410_gb300.build``).
"""
from __future__ import annotations

from . import capi
from .capi import FSA_F32, FSA_F64, FSA_KERNEL_BIHARMONIC3D, FSA_KERNEL_COULOMB3D, KERNELS, FsaError

_DT = {"f32": FSA_F32, "f64": FSA_F64, FSA_F32: FSA_F32, FSA_F64: FSA_F64}


def _torch_dtype(dt):
    import torch
    return torch.float32 if dt == FSA_F32 else torch.float64


def _cur_stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream()


class Plan:
    """A device-resident FSA plan: grid n (3 ints, or 2 for a plane kernel),
    box half-widths L, dtype 'f32' or 'f64', kernel 'coulomb3d',
    'biharmonic3d', 'poisson2d', 'coulomb2d' or 'biharmonic2d' (Table 1), or
    'ddi3d' (Sec. 5, Example 4: dipoles = (n, m), two 3-vectors, and
    ddi_derivative 'grid' or 'kernel'), or 'yukawa3d' / 'yukawa2d' (Example 4,
    kernel_param = lam, 0 selects 1).  eps = 0 picks min(1, R0/6).
    w_quadrature=1 takes W from the radial Gauss-Kronrod quadrature of
    Eq. Fourier-Symmetric instead of its closed form.  The spectrum is
    generated on construction unless generate=False."""

    def __init__(self, L, n, dtype="f32", eps=0.0, eps_tol=0.0, device=-1, generate=True, stream=None,
                 l2_chunk_mb=0, kernel="coulomb3d", dipoles=None, ddi_derivative="grid", kernel_param=0.0,
                 w_quadrature=0):
        self.dtype = _DT[dtype]
        self.n = tuple(int(x) for x in n)
        self.L = tuple(float(x) for x in L)
        self.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        if self.kernel == capi.FSA_KERNEL_DDI3D:
            if dipoles is None:
                raise ValueError("the ddi3d kernel needs dipoles=(n, m)")
            der = capi.DDI_DERIVATIVES[ddi_derivative] if isinstance(ddi_derivative, str) else int(ddi_derivative)
            self.handle = capi.fsa_plan_create_ddi3d(self.L, self.n, self.dtype, dipoles[0], dipoles[1], der, eps,
                                                     eps_tol, device)
        else:
            self.handle = capi.fsa_plan_create(self.kernel, len(self.n), self.L, self.n, self.dtype, eps, eps_tol,
                                               device, l2_chunk_mb, kernel_param, w_quadrature)
        if generate:
            self.generate(stream)

    @property
    def info(self):
        return capi.fsa_plan_info_get(self.handle)

    @property
    def eps(self):
        return self.info.eps

    def generate(self, stream=None):
        capi.fsa_tensor_generate(self.handle, _cur_stream(stream))

    def _check(self, t, what):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{what} must be a CUDA tensor")
        if t.dtype != _torch_dtype(self.dtype) or tuple(t.shape) != self.n or not t.is_contiguous():
            raise ValueError(f"{what} must be a contiguous {_torch_dtype(self.dtype)} tensor of shape {self.n}")

    def apply(self, rho, phi=None, stream=None):
        """phi = T * rho on the device; returns phi."""
        import torch
        self._check(rho, "rho")
        if phi is None:
            phi = torch.empty_like(rho)
        self._check(phi, "phi")
        capi.fsa_apply(self.handle, rho, phi, _cur_stream(stream))
        return phi

    def reserve(self, count):
        """Workspace for apply_many on up to count densities."""
        capi.fsa_plan_reserve(self.handle, count)

    def apply_many(self, rhos, phis=None, stream=None):
        """phi_k = T * rho_k for a list of densities in one launch sequence
        (reserve(len(rhos)) first); returns the list of outputs."""
        import torch
        for r in rhos:
            self._check(r, "rho")
        if phis is None:
            phis = [torch.empty_like(r) for r in rhos]
        for f in phis:
            self._check(f, "phi")
        capi.fsa_apply_many(self.handle, rhos, phis, _cur_stream(stream))
        return phis

    def apply_host(self, rho_host, phi_host, stream=None):
        """Host-buffer variant (copies inside); caller synchronises the stream."""
        capi.fsa_apply_host(self.handle, rho_host, phi_host, _cur_stream(stream))
        return phi_host

    def spectrum(self, stream=None):
        """A copy of the stored spectrum octant, shape (n0+1, n1+1, n2+1)."""
        import torch
        shp = tuple(x + 1 for x in self.n)
        out = torch.empty(shp, dtype=_torch_dtype(self.dtype), device="cuda")
        capi.fsa_plan_spectrum_copy(self.handle, out, out.numel() * out.element_size(), _cur_stream(stream))
        return out

    def close(self):
        if getattr(self, "handle", None):
            capi.fsa_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The continuous-batching serving loop (fsa_serve_*).  rho/phi are CUDA
    tensors owned by the caller until their ticket is DONE or FAILED."""

    def __init__(self, max_inflight=0, streams=0, hbm_fraction=0.0, hbm_budget_bytes=0, plan_cache_max=0,
                 queue_max=0, device=-1, policy=0):
        self.handle = capi.fsa_serve_create(max_inflight, streams, hbm_fraction, hbm_budget_bytes,
                                            plan_cache_max, queue_max, device, policy)

    def submit(self, L, n, dtype, rho, phi, eps=0.0, kernel="coulomb3d", kernel_param=0.0):
        k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        return capi.fsa_serve_submit(self.handle, L, n, _DT[dtype], rho, phi, eps, k, kernel_param)

    def poll(self, ticket, timeout=0.0):
        """(state, times); times has submit_s, admit_s, done_s, plan_hit, status."""
        return capi.fsa_serve_poll(self.handle, ticket, timeout)

    def wait(self, ticket, timeout=120.0):
        state, t = self.poll(ticket, timeout)
        if state in (capi.FSA_REQ_QUEUED, capi.FSA_REQ_RUNNING):
            raise FsaError(capi.FSA_ERR_TIMEOUT, f"request {ticket} not done after {timeout} s")
        if state != capi.FSA_REQ_DONE:
            raise FsaError(t.status, f"request {ticket} ended in state {state}")
        return t

    def stats(self):
        return capi.fsa_serve_stats_get(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            capi.fsa_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apply_batched(plans, rhos, phis, stream=None):
    """fsa_apply_batched over Plan objects and torch tensors."""
    capi.fsa_apply_batched([p.handle for p in plans], rhos, phis, _cur_stream(stream))
    return phis


__all__ = ["Plan", "Server", "apply_batched", "capi", "FsaError", "FSA_F32", "FSA_F64"]
