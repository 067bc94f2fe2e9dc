"""numpy float32 emulation of the CUDA forward recurrence (test helper).

Mirrors the FP32 evaluation order of the library's forward kernel (integer-
weight differences for L, 1 - G tabulated, K split in hi + lo, division by m)
so that the effect of FP32 wavefields alone can be measured on the CPU, with
the FP64 oracle supplying everything else.  Used only to explain tolerances.
"""
import numpy as np

import oracle

f32, f64 = np.float32, np.float64
A = [f32(8064), f32(-1008), f32(128), f32(-9)]


def _stencil(u):
    NZ, NX = u.shape
    p = np.zeros((NZ + 8, NX + 8), f32)
    p[4:-4, 4:-4] = u
    sz = np.zeros_like(u)
    sx = np.zeros_like(u)
    for k in range(1, 5):
        sz = sz + A[k - 1] * ((p[4 - k:4 - k + NZ, 4:-4] - u) + (p[4 + k:4 + k + NZ, 4:-4] - u))
        sx = sx + A[k - 1] * ((p[4:-4, 4 - k:4 - k + NX] - u) + (p[4:-4, 4 + k:4 + k + NX] - u))
    return sz + sx


def forward_fp32(g, m):
    """Traces (float64 array, CSR layout) of the float32 recurrence; dz == dx."""
    assert g.dz == g.dx
    nb = g.nb
    mp = oracle.extend(m, nb).astype(f32)
    dl = (1.0 - oracle.sponge(g.nz, g.nx, nb)).astype(f32)
    K = g.dt ** 2 / (5040.0 * g.dx ** 2)
    Kh = f32(K)
    Kl = f32(K - f64(Kh))
    wsp = (np.asarray(g.wavelet) * 5040.0 * g.dx / g.dz).astype(f32)
    out = []
    for s in range(g.S):
        u = np.zeros(mp.shape, f32)
        up = np.zeros_like(u)
        r0, r1 = g.rec_off[s], g.rec_off[s + 1]
        riz, rix = g.rec_iz[r0:r1] + nb, g.rec_ix[r0:r1] + nb
        tr = np.zeros((g.nt[s], r1 - r0))
        for n in range(g.nt[s]):
            T = _stencil(u)
            T[g.src_iz[s] + nb, g.src_ix[s] + nb] += wsp[n]
            y = T / mp
            wq = Kh * y + Kl * y
            gp = up - dl * up
            t = ((u - gp) + u) + wq
            up, u = u, t - dl * t
            tr[n] = u[riz, rix]
        out.append(tr.ravel())
    return np.concatenate(out)
