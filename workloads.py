"""Seeded synthetic densities shared by the tests, the bench and the oracle.

This module holds no step of the convolution method itself: it only builds
grids and evaluates analytic densities on them, in FP64, from seeded
parameters.  Both the CUDA path and the CPU oracle receive the arrays it
returns, so neither side generates its own inputs.

Grid convention (Sec. 2, the uniform mesh set; Sec. 2.4 for per-axis boxes):
axis j has n_j points x_{j,l} = h_j * l, l = -n_j/2 .. n_j/2 - 1, with
h_j = 2 L_j / n_j.  Array index i = l + n_j/2, C order, axis 2 fastest.

Workloads (all densities decay to round-off inside the box):
  * ``iso_gaussian``        exp(-|x|^2 / (2 w^2))                  (C1: w=1, [-8,8]^3)
  * ``gaussian_sum``        8 seeded isotropic Gaussians             (C2: [-16,16]^3)
  * ``aniso_gaussian``      exp(-sum_j x_j^2 / (2 s_j^2))            (cigar / pancake)
  * ``paper_case1``         exp(-(x^2 + y^2 + z^2/g^2) / sigma^2)    (Sec. 5, Example 1 Case I)
  * ``paper_case2``         -Laplacian of a Gaussian, plus a shifted copy (Example 1 Case II)
  * ``batch_requests`` / ``serve_requests``: seeded request mixes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Sizes the library supports per axis: even n = 2^a or 3 * 2^a (so 2n has
# only the radix factors 2 and 3 the FFT kernels implement), 4 <= n <= 512.
SUPPORTED_N = sorted({2 ** a for a in range(2, 10)} | {3 * 2 ** a for a in range(1, 8)})


def grid_axes(L, n):
    """Per-axis coordinates x_{j,l} = h_j * l, l = -n_j/2 .. n_j/2-1."""
    axes = []
    for Lj, nj in zip(L, n):
        h = 2.0 * Lj / nj
        axes.append(h * np.arange(-(nj // 2), nj - nj // 2, dtype=np.float64))
    return axes


def _sq(ax, c, s):
    return ((ax - c) / s) ** 2


@dataclass
class Gaussian:
    """a * exp(-sum_j (x_j - c_j)^2 / (2 s_j^2))."""
    amp: float
    center: tuple
    sigma: tuple

    def eval(self, L, n):
        x = grid_axes(L, n)
        e0 = _sq(x[0], self.center[0], self.sigma[0])[:, None, None]
        e1 = _sq(x[1], self.center[1], self.sigma[1])[None, :, None]
        e2 = _sq(x[2], self.center[2], self.sigma[2])[None, None, :]
        return self.amp * np.exp(-0.5 * (e0 + e1 + e2))


@dataclass
class Density:
    """A sum of Gaussians on a box [-L_j, L_j] with n_j points per axis."""
    L: tuple
    n: tuple
    terms: list = field(default_factory=list)
    eps: float = 1.0
    name: str = ""

    def rho(self):
        out = np.zeros(self.n, dtype=np.float64)
        for g in self.terms:
            out += g.eval(self.L, self.n)
        return out

    def rho_torch(self, dtype=None, device="cuda"):
        """The same density evaluated with torch on a device (for large
        request mixes whose host-side evaluation would be slow)."""
        import torch
        dtype = dtype or torch.float64
        out = torch.zeros(self.n, dtype=torch.float64, device=device)
        ax = [torch.from_numpy(a).to(device) for a in grid_axes(self.L, self.n)]
        for g in self.terms:
            e0 = ((ax[0] - g.center[0]) / g.sigma[0]) ** 2
            e1 = ((ax[1] - g.center[1]) / g.sigma[1]) ** 2
            e2 = ((ax[2] - g.center[2]) / g.sigma[2]) ** 2
            out += g.amp * torch.exp(-0.5 * (e0[:, None, None] + e1[None, :, None] + e2[None, None, :]))
        return out.to(dtype)

    def describe(self):
        return {"name": self.name, "L": list(self.L), "n": list(self.n), "eps": self.eps,
                "terms": [{"amp": g.amp, "center": list(g.center), "sigma": list(g.sigma)}
                          for g in self.terms]}


def iso_gaussian(L=8.0, n=32, w=1.0, eps=1.0):
    """C1: exp(-|x|^2/2) on [-8,8]^3 with 32^3 points."""
    return Density((L,) * 3, (n,) * 3, [Gaussian(1.0, (0.0, 0.0, 0.0), (w, w, w))], eps,
                   f"iso_gaussian_{n}")


def gaussian_sum(seed=2504, L=16.0, n=256, count=8, center_box=4.0,
                 width=(0.5, 1.5), amp=(-1.0, 1.0), eps=1.0, gamma=(1.0, 1.0, 1.0)):
    """C2: ``count`` isotropic Gaussians, centres U[-4,4]^3, widths U[0.5,1.5],
    amplitudes U[-1,1].  ``gamma`` > 1 on an axis compresses that axis: its box
    half-width, centres and widths are divided by gamma (cigar / pancake)."""
    rng = np.random.default_rng(seed)
    nn = (n,) * 3 if np.isscalar(n) else tuple(n)
    LL = tuple(L / g for g in gamma)
    terms = []
    for _ in range(count):
        c = rng.uniform(-center_box, center_box, 3)
        w = rng.uniform(*width)
        a = rng.uniform(*amp)
        terms.append(Gaussian(float(a), tuple(float(c[j] / gamma[j]) for j in range(3)),
                              tuple(float(w / gamma[j]) for j in range(3))))
    return Density(LL, nn, terms, eps, f"gaussian_sum_{count}_{nn[0]}x{nn[1]}x{nn[2]}_s{seed}")


@dataclass
class Plane:
    """A sum of isotropic Gaussians a exp(-|x-c|^2/(2 w^2)) on the plane box
    [-L_0, L_0] x [-L_1, L_1] with n_j points per axis (the d = 2 kernels)."""
    L: tuple
    n: tuple
    terms: list
    eps: float = 1.0
    name: str = ""

    def rho(self):
        x = grid_axes(self.L, self.n)
        out = np.zeros(self.n, dtype=np.float64)
        for a, c, w in self.terms:
            out += a * np.exp(-((x[0] - c[0])[:, None] ** 2 + (x[1] - c[1])[None, :] ** 2) / (2.0 * w * w))
        return out


def gaussian_sum_2d(seed=2504, L=16.0, n=512, count=8, center_box=4.0, width=(0.5, 1.5), amp=(-1.0, 1.0),
                    eps=1.0):
    """The plane analogue of C2: ``count`` Gaussians, centres U[-4,4]^2, widths
    U[0.5,1.5], amplitudes U[-1,1], on [-L, L]^2 with n x n points."""
    rng = np.random.default_rng(seed)
    terms = []
    for _ in range(count):
        c = rng.uniform(-center_box, center_box, 2)
        w = rng.uniform(*width)
        a = rng.uniform(*amp)
        terms.append((float(a), (float(c[0]), float(c[1])), float(w)))
    return Plane((L, L), (n, n), terms, eps, f"plane_gaussian_sum_{count}_{n}x{n}_s{seed}")


def aniso_gaussian(kind="cigar", gamma=8.0, eps=0.4):
    """C3: cigar exp(-(g^2 (x^2+y^2) + z^2)/2) on [-2,2]^2 x [-16,16], 128x128x512,
    or pancake exp(-(x^2+y^2+g^2 z^2)/2) on [-16,16]^2 x [-2,2], 512x512x128."""
    if kind == "cigar":
        L, n, s = (16.0 / gamma, 16.0 / gamma, 16.0), (128, 128, 512), (1 / gamma, 1 / gamma, 1.0)
    elif kind == "pancake":
        L, n, s = (16.0, 16.0, 16.0 / gamma), (512, 512, 128), (1.0, 1.0, 1 / gamma)
    else:
        raise ValueError(kind)
    return Density(L, n, [Gaussian(1.0, (0.0, 0.0, 0.0), s)], eps, f"{kind}_g{gamma:g}")


def scaled_density(d: Density, n):
    """Same analytic density and box on another grid (for convergence studies)."""
    nn = (n,) * 3 if np.isscalar(n) else tuple(n)
    return Density(d.L, nn, list(d.terms), d.eps, d.name + f"@{nn}")


def paper_case1(L=8.0, sigma2=0.8, gamma3=1.0, h_over_gamma=1.0):
    """Example 1 Case I (Sec. 5): exp(-(x^2+y^2+z^2/g^2)/sigma^2) on
    [-L,L]^2 x [-L g, L g] with h = g_j * h_over_gamma (same n per axis)."""
    s = math.sqrt(sigma2 / 2.0)
    Lj = (L, L, L * gamma3)
    n = int(round(2 * L / h_over_gamma))
    return Density(Lj, (n, n, n), [Gaussian(1.0, (0.0, 0.0, 0.0), (s, s, s * gamma3))],
                   1.0, f"case1_g{gamma3:g}_n{n}")


@dataclass
class Case2:
    """Example 1 Case II (Sec. 5): rho = rho0(x) + rho0(x - x0), rho0 = -Laplacian
    of Phi0 = exp(-(x^2+y^2+z^2/g^2)/sigma^2), on [-L,L]^2 x [-Lg, Lg]."""
    L: tuple
    n: tuple
    sigma2: float
    gamma3: float
    x0: tuple
    eps: float

    def rho(self):
        x = grid_axes(self.L, self.n)
        s2, g = self.sigma2, self.gamma3
        out = np.zeros(self.n)
        for c in ((0.0, 0.0, 0.0), self.x0):
            X = (x[0] - c[0])[:, None, None]
            Y = (x[1] - c[1])[None, :, None]
            Z = (x[2] - c[2])[None, None, :]
            phi0 = np.exp(-(X ** 2 + Y ** 2 + Z ** 2 / g ** 2) / s2)
            out += phi0 * (-4 * X ** 2 / s2 ** 2 - 4 * Y ** 2 / s2 ** 2
                           - 4 * Z ** 2 / (g ** 4 * s2 ** 2) + 4 / s2 + 2 / (g ** 2 * s2))
        return out


def paper_case2(L=12.0, sigma2=0.8, gamma3=1.0, h_over_gamma=0.125, eps=0.4, x0=(1.0, 1.0, 0.0)):
    n = int(round(2 * L / h_over_gamma))
    return Case2((L, L, L * gamma3), (n, n, n), sigma2, gamma3, tuple(x0), eps)


# ---- request mixes -------------------------------------------------------------

BATCH_N = (64, 96, 128, 192, 256)
BATCH_GAMMA = (1.0, 4.0, 8.0)


def default_eps(L):
    """Default FSA parameter: the largest eps <= 1 with R0/eps >= 6, where
    R0 = min_j 2 L_j (the App. B condition for 16-digit far-field accuracy)."""
    return min(1.0, min(2.0 * l for l in L) / 6.0)


def batch_requests(seed=2504, count=64, sizes=BATCH_N, gammas=BATCH_GAMMA):
    """C4: ``count`` 8-Gaussian densities; cubic n drawn from ``sizes``; gamma
    from ``gammas``; for gamma > 1 a coin flip picks cigar (x, y compressed) or
    pancake (z compressed).  Request i uses seed ``seed + i``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        g = float(rng.choice(gammas))
        if g > 1.0:
            gam = (g, g, 1.0) if rng.integers(2) == 0 else (1.0, 1.0, g)
        else:
            gam = (1.0, 1.0, 1.0)
        d = gaussian_sum(seed=seed + i, n=n, gamma=gam)
        d.eps = default_eps(d.L)
        out.append(d)
    return out


def round_serving_n(x):
    """Nearest supported n (2^a or 3*2^a) to x, within [32, 512]."""
    cand = [n for n in SUPPORTED_N if 32 <= n <= 512]
    return min(cand, key=lambda n: (abs(math.log(n / x)), n))


def serve_requests(seed=2504, count=10000, n_lo=32, n_hi=512, f64_share=0.2):
    """C5 request stream: n log-uniform in [32, 512] rounded to a supported size,
    isotropic [-16,16]^3 8-Gaussian densities, tier FP64 with probability
    ``f64_share`` else FP32.  Returns (n, dtype, seed) triples; the density of a
    request is ``gaussian_sum(seed=s, n=n)``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = round_serving_n(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))
        dt = "f64" if rng.uniform() < f64_share else "f32"
        out.append((n, dt, seed + 1 + i))
    return out


def poisson_arrivals(seed, count, rate_per_s):
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count))


# Dipole orientations of Example 4's 3-D DDI run (Sec. 5): n and m as printed.
DDI_N = (0.82778, 0.41505, -0.37751)
DDI_M = (0.3118, 0.9378, -0.15214)


def ddi_dipoles(seed):
    """A random pair of unit dipole orientations (n, m), for parity tests."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((2, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return tuple(v[0]), tuple(v[1])
