"""numpy float32 emulation of the CUDA forward recurrence (test helper).

Mirrors the FP32 evaluation of the library's step kernels, operation by
operation: the Laplacian as integer-weight differences to the centre cell,
accumulated from the smallest weight up through fused multiply-adds; the
model as the FP64-derived pair Wh + Wl of Wt = dt^2 / (5040 dx^2 m); the
sponge as x - (1 - G) x with 1 - G = dz + dx - dz dx from per-axis tables.
A fused multiply-add fma(a, b, c) of float32 operands is emulated in float64
(the product is exact there) with one rounding to float32.  Used only to explain tolerances
and the choice of evaluation order: the FP64 oracle supplies everything
else.

Besides the kernels' form, ``forward_fp32(form=...)`` emulates compensated
forms of the same recurrence that keep FP32 fields, to measure how far FP32
wavefields can go:
  "increment"    state (u^n, v^n = u^n - u^{n-1}):
                 v^{n+1} = -(1-G)^2 u^n + G^2 v^n + G W T,  u^{n+1} = u^n + v^{n+1}
                 (the rounding of the stored u no longer feeds the leap-frog's
                 secular mode);
  "compensated"  the increment form with u carried as an FP32 pair (hi, lo)
                 updated by an error-free sum, the stencil applied to both;
  "double_uv"    u and v both carried as FP32 pairs.
"""
import numpy as np

import oracle

f32, f64 = np.float32, np.float64
A = [f32(8064), f32(-1008), f32(128), f32(-9)]


def fma(a, b, c):
    """float32 fma with a single rounding (float64 product is exact)."""
    return (np.asarray(a, f64) * np.asarray(b, f64) + np.asarray(c, f64)).astype(f32)


def weighted_sum(d, order="small_first"):
    """sum_k A_k d_k: 'small_first' = the kernels' order (A4 d4 first, the
    dominant A1 d1 last through an fma); 'large_first' = A1 d1 rounded first;
    'plain' = separate roundings, left to right."""
    if order == "small_first":
        s = (A[3] * d[3]).astype(f32)
        for k in (2, 1, 0):
            s = fma(A[k], d[k], s)
    elif order == "large_first":
        s = (A[0] * d[0]).astype(f32)
        for k in (1, 2, 3):
            s = fma(A[k], d[k], s)
    else:
        s = (A[0] * d[0]).astype(f32)
        for k in (1, 2, 3):
            s = (s + (A[k] * d[k]).astype(f32)).astype(f32)
    return s


def stencil_T(u, rz=f32(1.0), order="small_first"):
    """T = rz S_z + S_x with S the integer-weight differences to the centre."""
    NZ, NX = u.shape
    p = np.zeros((NZ + 8, NX + 8), f32)
    p[4:-4, 4:-4] = u
    dz = [((p[4 - k:4 - k + NZ, 4:-4] - u) + (p[4 + k:4 + k + NZ, 4:-4] - u)).astype(f32) for k in range(1, 5)]
    dx = [((p[4:-4, 4 - k:4 - k + NX] - u) + (p[4:-4, 4 + k:4 + k + NX] - u)).astype(f32) for k in range(1, 5)]
    return fma(rz, weighted_sum(dz, order), weighted_sum(dx, order))


def two_sum(a, b):
    """Error-free sum of float32 arrays: s + e = a + b exactly (Knuth)."""
    s = (a + b).astype(f32)
    bb = (s - a).astype(f32)
    return s, ((a - (s - bb).astype(f32)).astype(f32) + (b - bb).astype(f32)).astype(f32)


def forward_fp32(g, m, order="small_first", form="kernel"):
    """Traces (float64 array, CSR layout) of the float32 recurrence."""
    nb = g.nb
    mp = oracle.extend(m, nb).astype(f64)
    G = oracle.sponge(g.nz, g.nx, nb)              # g(d_z) g(d_x); an interior column / row gives each factor
    dz = (1.0 - G[:, nb]).astype(f32)[:, None]     # the kernels' per-row and per-column tables of 1 - g
    dx = (1.0 - G[nb, :]).astype(f32)[None, :]
    ndG = fma(dz, dx, fma(dz, f32(-1.0), -dx))     # -(1 - G) = dz dx - (dz + dx), as the kernels form it
    Wt = g.dt ** 2 / (5040.0 * g.dx ** 2 * mp)
    wh = Wt.astype(f32)
    wl = (Wt - wh.astype(f64)).astype(f32)
    rz = f32(g.dx ** 2 / g.dz ** 2)
    wsp = (np.asarray(g.wavelet) * 5040.0 * g.dx / g.dz).astype(f32)
    # increment forms: -(1 - G)^2, G^2 and G per cell (FP64 tables rounded once)
    a_t = (-(1.0 - G) ** 2).astype(f32)
    b_t = (G * G).astype(f32)
    c_t = G.astype(f32)
    out = []
    for s in range(g.S):
        u = np.zeros(mp.shape, f32)
        up = np.zeros_like(u)       # kernel: u^{n-1}; increment forms: v^n
        ul = np.zeros_like(u)       # low parts of u (compensated) and of v (double_uv)
        vl = np.zeros_like(u)
        r0, r1 = g.rec_off[s], g.rec_off[s + 1]
        riz, rix = g.rec_iz[r0:r1] + nb, g.rec_ix[r0:r1] + nb
        tr = np.zeros((g.nt[s], r1 - r0))
        for n in range(g.nt[s]):
            T = stencil_T(u, rz, order)
            if form in ("compensated", "double_uv"):
                T = (T + stencil_T(ul, rz, order)).astype(f32)
            T[g.src_iz[s] + nb, g.src_ix[s] + nb] += wsp[n]
            wq = fma(wh, T, (wl * T).astype(f32))
            if form == "kernel":
                gp = fma(ndG, up, up)
                t = (((u - gp).astype(f32) + u).astype(f32) + wq).astype(f32)
                up, u = u, fma(ndG, t, t)
                tr[n] = u[riz, rix]
                continue
            if form == "double_uv":
                inc = fma(a_t, u, fma(b_t, vl, (c_t * wq).astype(f32)))
                bv = (b_t * up).astype(f32)
                vh, e1 = two_sum(bv, inc)
                vh, vl = two_sum(vh, (e1 + fma(b_t, up, -bv)).astype(f32))
                y = ((vh + ul).astype(f32) + vl).astype(f32)
            else:
                vh = fma(a_t, u, fma(b_t, up, (c_t * wq).astype(f32)))
                y = (vh + ul).astype(f32) if form == "compensated" else vh
            up = vh
            if form == "increment":
                u = (u + y).astype(f32)
                tr[n] = u[riz, rix]
            else:
                u, ul = two_sum(u, y)
                tr[n] = u[riz, rix].astype(f64) + ul[riz, rix].astype(f64)
        out.append(tr.ravel())
    return np.concatenate(out)
