"""aafwi_adjoint_gradient_host (host buffers in and out, copies inside the
call) gives bitwise the gradient and misfit of aafwi_adjoint_gradient on
device buffers, for FWI and LSRTM, and rejects missing arguments."""
import numpy as np
import pytest

from paper_2008_11778_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    from paper_2008_11778_gb300 import aafwi, build
    build.build()
    aafwi.load()
    assert torch.cuda.is_available()
    return aafwi


@pytest.mark.parametrize("mode", [0, 1], ids=["fwi", "lsrtm"])
def test_host_call_equals_device_call(A, orc, mode):
    import torch
    p = synth.small_problem(nz=40, nx=70, nb=10, nt=200, S=3)
    g = p.geom
    d = orc.forward(g, p.m_true).astype(np.float32)
    m = p.m_start.astype(np.float32)
    rho = np.random.default_rng(9).uniform(-0.1, 0.1, m.shape).astype(np.float32) if mode == 1 else None
    plan = A.Plan(g, 3000.0)
    dev = lambda a: None if a is None else torch.as_tensor(a, device="cuda")
    g_dev = torch.empty(m.shape, device="cuda")
    J_dev = plan.adjoint_gradient(mode, dev(m), dev(rho), dev(d), g_dev)
    host = lambda a: None if a is None else torch.as_tensor(a).pin_memory()
    g_host = torch.empty(m.shape).pin_memory()
    J_host = plan.adjoint_gradient_host(mode, host(m), host(rho), host(d), g_host)
    assert J_host == J_dev
    assert torch.equal(g_host, g_dev.cpu())
    g_page = torch.empty(m.shape)           # pageable host memory works too
    assert plan.adjoint_gradient_host(mode, torch.as_tensor(m), None if rho is None else torch.as_tensor(rho),
                                      torch.as_tensor(d), g_page) == J_dev
    assert torch.equal(g_page, g_host)
    if mode == 1:
        with pytest.raises(A.AafwiError):
            plan.adjoint_gradient_host(mode, host(m), None, host(d), g_host)
