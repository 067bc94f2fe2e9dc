"""The U-Net's 3x3 convolution GEMMs, one layer at a time, against the
oracle's float64 convolution (oracle/unet.py conv3 / conv3_back) on the same
BF16 operand values.  Products of BF16 values are exact in FP32, so the only
error is the FP32 accumulation: element by element |y - ref| stays within
(K/16 + 1) 2^-22 times the sum of the absolute terms (S, the same
convolution of |x| and |w|), K = 9 C, while one wrong tap, channel, padding
cell or split in a sum of K terms moves an output by about S / K.

Shapes: the production network's layers (C = 32 on 96 x 256, the 8C bottom,
the 400-wide evaluation grid), ragged tiles (positions not a multiple of
the 128-row tile, N not a multiple of 16, two N tiles), channel stages split
over CTAs (the deep layers), and the gathered path (channels not 16 times a
power of two)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    from paper_2008_11778_gb300 import aafwi, build
    build.build()
    aafwi.load()
    assert torch.cuda.is_available()
    return aafwi


def bf16_pair(rng, shape, scale=1.0):
    """(device BF16 tensor, the same values in float64)."""
    import torch
    t = torch.as_tensor((scale * rng.standard_normal(shape)).astype(np.float32)).to(torch.bfloat16)
    return t.cuda().contiguous(), t.to(torch.float64).numpy()


SHAPES = [
    # B, H, W, Cin, Cout
    (2, 96, 256, 32, 32),      # level 0 of the production network
    (2, 48, 128, 64, 64),      # level 1
    (16, 12, 32, 256, 256),    # bottom, training batch (split-K forward)
    (1, 19, 50, 128, 256),     # bottom of the 152 x 400 evaluation grid
    (1, 24, 64, 256, 128),     # decoder level 2 first conv (largest window)
    (3, 5, 7, 16, 48),         # ragged: 3 x 7 x 9 positions, N = 48
    (2, 8, 8, 48, 16),         # C = 48: gathered (channels not 16 times a power of two)
    (1, 3, 4, 32, 8),          # N = 8 < 16, fewer positions than one tile
    (2, 6, 10, 32, 272),       # two N tiles (256 + 16)
    (2, 16, 32, 8, 16),        # gathered path (C = 8)
    (2, 16, 32, 2, 32),        # gathered path, the network's first layer
]


def bound(K, S):
    return (K / 16 + 1) * 2.0 ** -22 * S + 1e-30


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_conv3_forward_matches_oracle(A, shape):
    from oracle import unet as U
    B, H, W, Cin, Cout = shape
    rng = np.random.default_rng(sum(shape))
    x, xh = bf16_pair(rng, (B, H, W, Cin))
    w, wh = bf16_pair(rng, (Cout, 3, 3, Cin), 0.2)
    out, s = A.unet_conv3x3(A.CONV3_FWD, x, w, B, H, W, Cin, Cout)
    y = out.double().sum(0).cpu().numpy().reshape(B, H, W, Cout)
    ref = U.conv3(xh, wh, np.zeros(Cout))
    S = U.conv3(np.abs(xh), np.abs(wh), np.zeros(Cout))
    err = np.abs(y - ref)
    assert (err <= bound(9 * Cin, S)).all(), (s, float((err / (S + 1e-30)).max()))


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_conv3_data_gradient_matches_oracle(A, shape):
    from oracle import unet as U
    B, H, W, Cin, Cout = shape
    rng = np.random.default_rng(100 + sum(shape))
    dz, dzh = bf16_pair(rng, (B, H, W, Cout))
    w, wh = bf16_pair(rng, (Cout, 3, 3, Cin), 0.2)
    wt = w.permute(3, 1, 2, 0).contiguous()            # [Cin][3][3][Cout]
    out, s = A.unet_conv3x3(A.CONV3_DGRAD, dz, wt, B, H, W, Cin, Cout)
    gx = out.double().sum(0).cpu().numpy().reshape(B, H, W, Cin)
    xz = np.zeros((B, H, W, Cin))
    ref = U.conv3_back(xz, wh, dzh)[0]
    S = U.conv3_back(xz, np.abs(wh), np.abs(dzh))[0]
    err = np.abs(gx - ref)
    assert (err <= bound(9 * Cout, S)).all(), (s, float((err / (S + 1e-30)).max()))


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_conv3_weight_gradient_matches_oracle(A, shape):
    from oracle import unet as U
    B, H, W, Cin, Cout = shape
    rng = np.random.default_rng(200 + sum(shape))
    x, xh = bf16_pair(rng, (B, H, W, Cin))
    dz, dzh = bf16_pair(rng, (B, H, W, Cout))
    out, s = A.unet_conv3x3(A.CONV3_WGRAD, dz, x, B, H, W, Cin, Cout)
    dw = out.double().sum(0).cpu().numpy().reshape(Cout, 3, 3, Cin)
    w0 = np.zeros((Cout, 3, 3, Cin))
    ref = U.conv3_back(xh, w0, dzh)[1]
    S = U.conv3_back(np.abs(xh), w0, np.abs(dzh))[1]
    err = np.abs(dw - ref)
    assert (err <= bound(B * H * W, S)).all(), (s, float((err / (S + 1e-30)).max()))


def test_conv3_forward_split_slices_sum_to_one_result(A):
    """A forward forced to 1 and to 4 K splits: the same result within the
    accumulation bound (the splits partition the channel stages; with one
    split a CTA runs all eight stages through its two buffers)."""
    B, H, W, Cin, Cout = 2, 24, 64, 256, 128
    rng = np.random.default_rng(7)
    x, _ = bf16_pair(rng, (B, H, W, Cin))
    w, _ = bf16_pair(rng, (Cout, 3, 3, Cin), 0.2)
    o1, s1 = A.unet_conv3x3(A.CONV3_FWD, x, w, B, H, W, Cin, Cout, splits=1)
    o4, s4 = A.unet_conv3x3(A.CONV3_FWD, x, w, B, H, W, Cin, Cout, splits=4)
    assert (s1, s4) == (1, 4)
    y1, y4 = o1.double().sum(0), o4.double().sum(0)
    assert float((y1 - y4).abs().max()) <= 1e-5 * float(y1.abs().max())


def test_conv3_weight_gradient_one_span_equals_many(A):
    """The windowed weight gradient with one position span (all stages in
    one CTA, two buffers in turn) and with its own split: the same result."""
    B, H, W, Cin, Cout = 2, 24, 64, 64, 64
    rng = np.random.default_rng(9)
    x, _ = bf16_pair(rng, (B, H, W, Cin))
    dz, _ = bf16_pair(rng, (B, H, W, Cout))
    o1, s1 = A.unet_conv3x3(A.CONV3_WGRAD, dz, x, B, H, W, Cin, Cout, splits=1)
    on, sn = A.unet_conv3x3(A.CONV3_WGRAD, dz, x, B, H, W, Cin, Cout)
    assert s1 == 1 and sn > 1
    y1, yn = o1.double().sum(0), on.double().sum(0)
    assert float((y1 - yn).abs().max()) <= 1e-5 * float(y1.abs().max())


def test_conv3_rejects_bad_arguments(A):
    import torch
    x = torch.zeros(16, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(A.AafwiError):
        A.unet_conv3x3(7, x, x, 1, 2, 2, 2, 2)
    with pytest.raises(A.AafwiError):
        A.unet_conv3x3(A.CONV3_FWD, x, x, 0, 2, 2, 2, 2)
