"""The BF16 tensor-core U-Net runtime against its CPU reference (oracle/unet.py
in its BF16-rounding mode): forward output, loss and parameter gradient."""
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


def rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def case(seed, B=2, H=16, W=32, C=16):
    from oracle import unet as U
    rng = np.random.default_rng(seed)
    p = U.init_params(C, seed)
    x = rng.standard_normal((B, 2, H, W)).astype(np.float32)
    t = (0.1 * rng.standard_normal((B, H, W))).astype(np.float32)
    return p, x, t


@pytest.mark.parametrize("C", [8, 16])
def test_unet_forward_matches_reference(A, C):
    import torch
    from oracle import unet as U
    p, x, _ = case(1, C=C)
    net = A.UNet(2, 16, 32, C)
    assert net.nparam == U.param_count(C)
    net.set_params(p)
    y = net.forward(torch.as_tensor(x, device="cuda")).cpu().numpy()
    ref = U.forward(p, x, C)
    assert rel(y, ref) < 2e-3
    exact = U.forward(p, x, C, exact=True)
    assert rel(y, exact) < 5e-2          # BF16 activations against float64


def test_unet_gradient_matches_reference(A):
    import torch
    from oracle import unet as U
    C = 16
    p, x, t = case(2, C=C)
    net = A.UNet(2, 16, 32, C)
    net.set_params(p)
    g = torch.empty(net.nparam, device="cuda")
    L = net.loss_grad(torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"), g)
    Lr, gr = U.loss_grad(p, x, t, C)
    assert L == pytest.approx(Lr, rel=1e-3)
    g = g.cpu().numpy()
    assert rel(g, gr) < 2e-2
    # every layer's slice, weights and bias
    o = 0
    for kind, ci, co in U.layers(C):
        nw = (9 if kind == "c3" else 4) * ci * co
        assert rel(g[o:o + nw], gr[o:o + nw]) < 5e-2, (kind, ci, co)
        o += nw + co


def test_unet_training_reduces_loss(A):
    import torch
    from oracle import unet as U
    C = 16
    p, x, t = case(3, B=4, C=C)
    t = np.tanh(x[:, 0] + 0.5 * x[:, 1]).astype(np.float32)      # a learnable target
    net = A.UNet(4, 16, 32, C)
    net.set_params(p)
    xd, td = torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda")
    L0 = net.loss_grad(xd, td)
    for _ in range(60):
        L = net.train_step(xd, td, 2e-3)
    assert L < 0.3 * L0
    assert np.isfinite(net.get_params()).all()


@pytest.fixture(scope="module")
def production_case():
    """The production network (C = 32) on a batch of the training shape
    (2 x 96 x 256): split-K weight gradients and 16-byte channel gathers run
    as in training.  Reference: the oracle in its BF16-rounding mode and in
    FP64."""
    from oracle import unet as U
    C = 32
    rng = np.random.default_rng(17)
    p = U.init_params(C, 17)
    x = rng.standard_normal((2, 2, 96, 256)).astype(np.float32)
    t = (0.1 * rng.standard_normal((2, 96, 256))).astype(np.float32)
    return C, p, x, t, U.loss_grad(p, x, t, C), U.loss_grad(p, x, t, C, exact=True)


def test_unet_production_shape_forward(A, production_case):
    """Forward of the C = 32 network on a 2 x 96 x 256 batch: the runtime sits
    within a quarter of the BF16 quantisation error (the BF16 reference
    against FP64) of the BF16 reference."""
    import torch
    from oracle import unet as U
    C, p, x, _, _, _ = production_case
    net = A.UNet(2, 96, 256, C)
    net.set_params(p)
    y = net.forward(torch.as_tensor(x, device="cuda")).cpu().numpy()
    ref, exact = U.forward(p, x, C), U.forward(p, x, C, exact=True)
    q = rel(ref, exact)                  # what BF16 activations cost
    assert rel(y, ref) < 0.25 * q
    net.close()


def test_unet_production_shape_gradient_per_layer(A, production_case):
    """Loss gradient of the C = 32 network on a 2 x 96 x 256 batch, layer by
    layer: each weight and bias slice of the runtime lies within half of that
    slice's BF16 quantisation error (BF16 reference against FP64) of the BF16
    reference (the runtime accumulates in FP32 where the reference uses FP64,
    so a BF16 rounding or a ReLU mask can flip where a value sits on the
    boundary)."""
    import torch
    from oracle import unet as U
    C, p, x, t, (Lr, gr), (Le, ge) = production_case
    net = A.UNet(2, 96, 256, C)
    net.set_params(p)
    g = torch.empty(net.nparam, device="cuda")
    L = net.loss_grad(torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"), g)
    g = g.cpu().numpy()
    assert abs(L - Lr) <= 0.25 * abs(Lr - Le) + 1e-6 * abs(Lr)
    o = 0
    for kind, ci, co in U.layers(C):
        nw = (9 if kind == "c3" else 4) * ci * co
        for a, b in ((o, o + nw), (o + nw, o + nw + co)):
            q = rel(gr[a:b], ge[a:b])
            assert rel(g[a:b], gr[a:b]) < 0.5 * q, (kind, ci, co, a == o, rel(g[a:b], gr[a:b]), q)
        o += nw + co
    assert rel(g[o:], gr[o:]) < 0.5 * rel(gr[o:], ge[o:])      # the 1x1 head
    net.close()
