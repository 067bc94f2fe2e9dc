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
