"""CPU reference of the learned preconditioner's U-Net (numpy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The network is not part
of the paper; this module fixes what the CUDA runtime must compute: the
architecture, the parameter layout, the forward pass, the loss and the
hand-written backward pass.

Two precisions:
  * exact=True : float64 everywhere (pinned by finite differences and a brute
    force convolution in the tests);
  * exact=False: the rounding points of the BF16 tensor-core runtime --
    inputs, weights and every stored activation rounded to BF16
    (round-to-nearest-even), activation gradients rounded to BF16 where they
    become a GEMM operand, sums in float64 (the runtime sums in FP32).

Layout: activations NHWC [B][H][W][C]; 3x3 weights [Cout][3][3][Cin]
(cross-correlation, zero padding 1); 2x2 stride-2 transposed conv weights
[Cin][2][2][Cout], output child (2y+i, 2x+j) of input pixel (y, x); maxpool
2x2 routes the gradient to the first maximum in the order (0,0), (0,1),
(1,0), (1,1); loss 1/(2N) sum (y - t)^2 over the N output pixels.
"""
import numpy as np


def bf16(a):
    """Round float32 values to BF16 (round to nearest, ties to even), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).reshape(a.shape)


def layers(C):
    """(kind, Cin, Cout) of the 17 convolutions in network / parameter order."""
    L = [("c3", 2, C), ("c3", C, C), ("c3", C, 2 * C), ("c3", 2 * C, 2 * C),
         ("c3", 2 * C, 4 * C), ("c3", 4 * C, 4 * C), ("c3", 4 * C, 8 * C), ("c3", 8 * C, 8 * C)]
    for l in (2, 1, 0):
        L += [("up", C << (l + 1), C << l), ("c3", C << (l + 1), C << l), ("c3", C << l, C << l)]
    return L


def unpack(params, C):
    """Split the flat parameter vector into per-layer (w, b) and the head."""
    out, o = [], 0
    for kind, ci, co in layers(C):
        nw = 9 * ci * co if kind == "c3" else 4 * ci * co
        w = params[o:o + nw].reshape((co, 3, 3, ci) if kind == "c3" else (ci, 2, 2, co))
        o += nw
        b = params[o:o + co]
        o += co
        out.append((kind, w, b))
    hw = params[o:o + C]
    hb = params[o + C:o + C + 1]
    assert o + C + 1 == params.size
    return out, hw, hb


def param_count(C):
    n = 0
    for kind, ci, co in layers(C):
        n += (9 if kind == "c3" else 4) * ci * co + co
    return n + C + 1


def init_params(C, seed):
    """He-normal weights, zero biases, small head (seeded input generator)."""
    rng = np.random.default_rng(seed)
    parts = []
    for kind, ci, co in layers(C):
        fan = 9 * ci if kind == "c3" else ci
        nw = (9 if kind == "c3" else 4) * ci * co
        parts += [rng.standard_normal(nw) * np.sqrt(2.0 / fan), np.zeros(co)]
    parts += [rng.standard_normal(C) * 0.1 / np.sqrt(C), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


# ---------------------------------------------------------------- operators

def conv3(x, w, b):
    """y[b,i,j,o] = sum_{ky,kx,c} x[b,i+ky-1,j+kx-1,c] w[o,ky,kx,c] + b[o]."""
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, W, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            y += xp[:, ky:ky + H, kx:kx + W, :] @ w[:, ky, kx, :].T
    return y + b


def conv3_back(x, w, dz):
    """Gradients of conv3 w.r.t. x and w given dz = dL/dy."""
    B, H, W, Ci = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp, dtype=np.float64)
    dw = np.zeros(w.shape)
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + H, kx:kx + W, :] += dz @ w[:, ky, kx, :]
            dw[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", dz, xp[:, ky:ky + H, kx:kx + W, :])
    return dxp[:, 1:-1, 1:-1, :], dw


def up2(x, w, b):
    """2x2 stride-2 transposed conv: y[b,2i+p,2j+q,o] = sum_c x[b,i,j,c] w[c,p,q,o] + b[o]."""
    B, H, W, _ = x.shape
    y = np.zeros((B, 2 * H, 2 * W, w.shape[3]))
    for p in range(2):
        for q in range(2):
            y[:, p::2, q::2, :] = x @ w[:, p, q, :]
    return y + b


def up2_back(x, w, dy):
    dx = np.zeros(x.shape)
    dw = np.zeros(w.shape)
    for p in range(2):
        for q in range(2):
            g = dy[:, p::2, q::2, :]
            dx += g @ w[:, p, q, :].T
            dw[:, p, q, :] = np.einsum("bhwc,bhwo->co", x, g)
    return dx, dw


def maxpool(x):
    """2x2 max pool and the index (0..3, first maximum) of each winner."""
    c = np.stack([x[:, 0::2, 0::2], x[:, 0::2, 1::2], x[:, 1::2, 0::2], x[:, 1::2, 1::2]])
    idx = np.argmax(c, axis=0)       # argmax returns the first maximum
    return np.take_along_axis(c, idx[None], 0)[0], idx


def maxpool_back(dy, idx, shape):
    dx = np.zeros(shape)
    for k, (p, q) in enumerate(((0, 0), (0, 1), (1, 0), (1, 1))):
        dx[:, p::2, q::2] += np.where(idx == k, dy, 0.0)
    return dx


# ------------------------------------------------------------------ network

def forward(params, x_nchw, C, exact=False, keep=False):
    """Network output [B][H][W] for input [B][2][H][W]."""
    R = (lambda a: np.asarray(a, dtype=np.float64)) if exact else (lambda a: bf16(a).astype(np.float64))
    P = np.asarray(params, dtype=np.float64 if exact else np.float32)
    Ls, hw, hb = unpack(P, C)
    Wr = [(k, R(w), np.asarray(b, dtype=np.float64)) for k, w, b in Ls]
    x = R(np.transpose(np.asarray(x_nchw, dtype=np.float64 if exact else np.float32), (0, 2, 3, 1)))
    t = {"x": x}
    li = 0
    skips, h = [], x
    for l in range(3):
        a = R(np.maximum(conv3(h, Wr[li][1], Wr[li][2]), 0)); li += 1
        s = R(np.maximum(conv3(a, Wr[li][1], Wr[li][2]), 0)); li += 1
        h, idx = maxpool(s)
        t["ea%d" % l], t["eb%d" % l], t["idx%d" % l], t["pool%d" % l] = a, s, idx, h
        skips.append(s)
    a = R(np.maximum(conv3(h, Wr[li][1], Wr[li][2]), 0)); li += 1
    h = R(np.maximum(conv3(a, Wr[li][1], Wr[li][2]), 0)); li += 1
    t["ba"], t["bb"] = a, h
    for l in (2, 1, 0):
        u = R(up2(h, Wr[li][1], Wr[li][2])); li += 1
        c = np.concatenate([u, skips[l]], axis=-1)
        a = R(np.maximum(conv3(c, Wr[li][1], Wr[li][2]), 0)); li += 1
        h = R(np.maximum(conv3(a, Wr[li][1], Wr[li][2]), 0)); li += 1
        t["cat%d" % l], t["da%d" % l], t["db%d" % l] = c, a, h
    y = h @ R(hw) + float(hb[0])
    t["hw"] = R(hw)
    t["W"] = Wr
    return (y, t) if keep else y


def loss_grad(params, x_nchw, target, C, exact=False):
    """(loss, gradient of the flat parameter vector)."""
    y, t = forward(params, x_nchw, C, exact, keep=True)
    Rg = (lambda a: a) if exact else (lambda a: bf16(a).astype(np.float64))
    N = y.size
    d = y - np.asarray(target, dtype=np.float64)
    loss = 0.5 * float((d * d).sum()) / N
    dout = d / N
    if not exact:
        dout = dout.astype(np.float32).astype(np.float64)
    Wr = t["W"]
    grads = [None] * len(Wr)
    g_hw = np.einsum("bhw,bhwc->c", dout, t["db0"])
    g_hb = np.array([dout.sum()])
    g = dout[..., None] * t["hw"]                 # gradient of db0 (FP32 in the runtime)

    def c3back(li, x, y, g):
        dz = np.where(y > 0, Rg(g), 0.0)
        dx, dw = conv3_back(x, Wr[li][1], dz)
        grads[li] = (dw, dz.sum(axis=(0, 1, 2)))
        return dx

    li = 16
    gsk = {}
    for l in (0, 1, 2):
        g = c3back(li, t["da%d" % l], t["db%d" % l], g); li -= 1
        g = c3back(li, t["cat%d" % l], t["da%d" % l], g); li -= 1
        Cv = g.shape[-1] // 2
        gu, gsk[l] = Rg(g[..., :Cv]), g[..., Cv:]
        xin = t["bb"] if l == 2 else t["db%d" % (l + 1)]
        dx, dw = up2_back(xin, Wr[li][1], gu)
        grads[li] = (dw, gu.sum(axis=(0, 1, 2))); li -= 1
        g = dx
    g = c3back(li, t["ba"], t["bb"], g); li -= 1
    g = c3back(li, t["pool2"], t["ba"], g); li -= 1
    for l in (2, 1, 0):
        gs = maxpool_back(g, t["idx%d" % l], t["eb%d" % l].shape) + gsk[l]
        g = c3back(li, t["ea%d" % l], t["eb%d" % l], gs); li -= 1
        xin = t["x"] if l == 0 else t["pool%d" % (l - 1)]
        g = c3back(li, xin, t["ea%d" % l], g); li -= 1
    flat = []
    for dw, db in grads:
        flat += [dw.ravel(), db.ravel()]
    flat += [g_hw, g_hb]
    return loss, np.concatenate(flat)
