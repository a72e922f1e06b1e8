"""Host-side check of the fused outer pass pairs' index maps (passes5.cuh).

The cluster kernels move data between CTAs through distributed shared memory,
and compute-sanitizer is not available, so their address arithmetic is
checked here on the CPU for every configuration the library registers
(fsa_fused_configs): each CTA's remote stores are replayed with the kernels'
own formulas (owner CTA, byte offset, alignment), every receive slot and every
output element must be written exactly once and in bounds, the Hermitian split
of line 0 must take its mirror value from the right thread and register, and
the data flow, with numpy's FFTs standing in for the register transforms, must
give the same Y (forward) and Phi (inverse) as plain transforms.
"""
import numpy as np
import pytest

# Two-step plans M = R1 x R2 of the lengths with fused pairs (fft_reg.cuh: Plan2For);
# threads per line T = R1.
PLANS = {64: (8, 8), 128: (8, 16), 256: (16, 16), 384: (16, 24), 512: (16, 32)}


def geometry(M, CS, NT):
    """FusedGeo: the same quantities, the same static checks."""
    R1, R2 = PLANS[M]
    T = R1
    n0 = n2 = M // 2
    g = dict(R1=R1, R2=R2, T=T, n0=n0, n2=n2, CW=n2 // CS, W0=NT // T, LR=n0 // CS, W2=NT // T)
    g["LW"] = g["CW"] // 2
    g["R0"] = g["LW"] // g["W0"]
    g["RR"] = g["LR"] // g["W2"]
    assert NT % T == 0 and 32 % T == 0
    assert n2 % (2 * CS) == 0 and g["LW"] % g["W0"] == 0 and g["R0"] >= 1
    assert n0 % CS == 0 and g["LR"] % g["W2"] == 0 and g["RR"] >= 1
    pitch2 = R1 * (R2 + 1)
    g["XCH"] = max(M * g["W0"], g["W2"] * pitch2) * 8
    g["RCV_F"] = g["LR"] * n2 * 8
    g["RCV_I"] = (n0 + 1) * g["CW"] * 8
    return g


def forward(rho, M, CS, NT):
    g = geometry(M, CS, NT)
    n0, n2, CW, W0, T, R1, R2 = (g[k] for k in ("n0", "n2", "CW", "W0", "T", "R1", "R2"))
    n1 = rho.shape[1]
    Y = np.full((n0 + 1, n1, M), np.nan + 0j)
    for i1 in range(n1):
        rcv = [np.full(g["RCV_F"] // 8, np.nan + 0j) for _ in range(CS)]
        # phase 1: column pairs along axis 0, rows to their owners
        for rank in range(CS):
            for rd in range(g["R0"]):
                for l in range(W0):
                    i2 = rank * CW + 2 * (rd * W0 + l)
                    z = np.zeros(M, complex)
                    z[:n0] = rho[:, i1, i2] + 1j * rho[:, i1, i2 + 1]
                    Z = np.fft.fft(z)
                    for u in range(T):
                        for k in range(u, n0, T):
                            if k == 0:
                                zk, zh = Z[0], Z[n0]
                                v = (complex(zk.real, zh.real), complex(zk.imag, zh.imag))
                            else:
                                zk, zm = Z[k], Z[M - k]
                                v = (0.5 * (zk + np.conj(zm)), (zk - np.conj(zm)) / 2j)
                            off, owner = ((k // CS) * n2 + i2) * 8, k % CS
                            assert 0 <= owner < CS and off % 16 == 0 and off + 16 <= g["RCV_F"]
                            a = off // 8
                            assert np.isnan(rcv[owner][a]) and np.isnan(rcv[owner][a + 1])
                            rcv[owner][a], rcv[owner][a + 1] = v
        assert not any(np.isnan(r).any() for r in rcv)
        # phase 2: rows along axis 2; line 0 split by Hermitian symmetry
        for rank in range(CS):
            for rd in range(g["RR"]):
                for l in range(g["W2"]):
                    j = rd * g["W2"] + l
                    k0 = rank + CS * j
                    assert k0 < n0
                    line = np.zeros(M, complex)
                    line[:n2] = rcv[rank][j * n2:(j + 1) * n2]
                    Z = np.fft.fft(line)
                    if k0 != 0:
                        Y[k0, i1] = Z
                        continue
                    # the warp holding line 0: CTA rank 0, round 0, threads < 32
                    assert rank == 0 and rd == 0 and (l + 1) * T <= 32
                    for u in range(T):
                        for s in range(R2):
                            k2 = u + R1 * s
                            km = R1 * ((R2 - s) % R2) if u == 0 else (T - u) % T + R1 * (R2 - 1 - s)
                            assert km == (M - k2) % M
                            z, m = Z[k2], Z[km]
                            Y[0, i1, k2] = 0.5 * (z + np.conj(m))
                            Y[n0, i1, k2] = (z - np.conj(m)) / 2j
    return Y


def inverse(Yin, M, CS, NT):
    g = geometry(M, CS, NT)
    n0, n2, CW, W0, T, R1, R2 = (g[k] for k in ("n0", "n2", "CW", "W0", "T", "R1", "R2"))
    n1 = Yin.shape[1]
    phi = np.full((n0, n1, n2), np.nan)
    for i1 in range(n1):
        rcv = [np.full(g["RCV_I"] // 8, np.nan + 0j) for _ in range(CS)]
        # phase A: rows along axis 2 (inverse, cropped), values to the column owners
        for rank in range(CS):
            for rd in range(g["RR"]):
                for l in range(g["W2"]):
                    k0 = rank + CS * (rd * g["W2"] + l)
                    b = Yin[0, i1] + 1j * Yin[n0, i1] if k0 == 0 else Yin[k0, i1]
                    x = np.fft.ifft(b) * M
                    for p in range(n2):
                        owner, cl = p // CW, p % CW
                        assert 0 <= owner < CS
                        stores = ([(cl * 8, x[p].real), ((n0 * CW + cl) * 8, x[p].imag)] if k0 == 0
                                  else [((k0 * CW + cl) * 8, x[p])])
                        for off, val in stores:
                            assert off % 8 == 0 and off + 8 <= g["RCV_I"]
                            assert np.isnan(rcv[owner][off // 8])
                            rcv[owner][off // 8] = val
        assert not any(np.isnan(r).any() for r in rcv)
        # phase B: C2R along axis 0 of each CTA's column pairs, crop to i0 < n0
        for rank in range(CS):
            for rd in range(g["R0"]):
                for l in range(W0):
                    cl = 2 * (rd * W0 + l)
                    c = rank * CW + cl
                    Z = np.zeros(M, complex)
                    for u in range(T):
                        for s in range(R2):
                            k = u + R1 * s
                            kk = k if k <= n0 else M - k
                            off = (kk * CW + cl) * 8
                            assert off % 16 == 0 and off + 16 <= g["RCV_I"]
                            a, bb = rcv[rank][kk * CW + cl], rcv[rank][kk * CW + cl + 1]
                            Z[k] = (complex(a.real - bb.imag, a.imag + bb.real) if k <= n0
                                    else complex(a.real + bb.imag, bb.real - a.imag))
                    z = np.fft.ifft(Z) * M
                    for p in range(n0):
                        assert np.isnan(phi[p, i1, c]) and np.isnan(phi[p, i1, c + 1])
                        phi[p, i1, c], phi[p, i1, c + 1] = z[p].real, z[p].imag
    return phi


def registered():
    from paper_2504_19410_gb300 import capi
    return [(M, cs, nt) for M in sorted(PLANS) for cs, nt in capi.fsa_fused_configs(M)]


@pytest.fixture(scope="module")
def configs():
    import __graft_entry__ as g
    g.build()
    c = registered()
    assert {M for M, _, _ in c} == set(PLANS)
    return c


def test_every_registered_configuration(configs):
    rng = np.random.default_rng(11)
    for M, CS, NT in configs:
        g = geometry(M, CS, NT)
        assert g["RCV_F"] + g["XCH"] <= 227 * 1024 and g["RCV_I"] + g["XCH"] <= 227 * 1024
        n = M // 2
        n1 = 2 if M <= 256 else 1
        rho = rng.standard_normal((n, n1, n))
        Y = forward(rho, M, CS, NT)
        want = np.fft.fft(np.fft.fft(rho, n=M, axis=0)[: n + 1], n=M, axis=2)
        assert np.abs(Y - want).max() <= 1e-12 * np.abs(want).max(), (M, CS, NT)
        # inverse input: the half spectrum of a real field (rows k0 = 0, n0 Hermitian in k2)
        field = rng.standard_normal((M, n1, M))
        G = np.fft.fft(np.fft.fft(field, axis=0), axis=2)[: n + 1]
        phi = inverse(G, M, CS, NT)
        ref = M * M * field[:n, :, :n]
        assert np.abs(phi - ref).max() <= 1e-12 * np.abs(ref).max(), (M, CS, NT)
