"""torch.autograd wrappers: backward passes are the library's adjoint-state
kernels, checked against the FP64 oracle and by finite differences."""
import numpy as np
import pytest

from paper_2008_11778_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    from paper_2008_11778_gb300 import aafwi, build
    build.build()
    aafwi.load()
    return torch


def rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def setup(T, orc):
    from paper_2008_11778_gb300 import aafwi
    p = synth.small_problem(nz=48, nx=120, nb=12, nt=300, S=3)
    plan = aafwi.Plan(p.geom, c_max=3000.0)
    d_obs = orc.forward(p.geom, p.m_true).astype(np.float32)
    return p, plan, T.as_tensor(d_obs, device="cuda")


def test_fwi_misfit_backward_is_the_oracle_gradient(T, orc):
    from paper_2008_11778_gb300 import autograd as ag
    p, plan, d_obs = setup(T, orc)
    m = T.as_tensor(p.m_start.astype(np.float32), device="cuda").requires_grad_(True)
    J = ag.fwi_misfit(m, plan, d_obs)
    (3.0 * J).backward()
    J_ref, g_ref = orc.fwi_gradient(p.geom, p.m_start.astype(np.float32), d_obs.cpu().numpy())
    assert float(J) == pytest.approx(J_ref, rel=1e-5)
    assert rel(m.grad.cpu().numpy() / 3.0, g_ref) < 1e-4


def test_fwi_misfit_central_differences(T, orc):
    from paper_2008_11778_gb300 import autograd as ag
    p, plan, d_obs = setup(T, orc)
    m0 = T.as_tensor(p.m_start.astype(np.float32), device="cuda")
    m = m0.clone().requires_grad_(True)
    ag.fwi_misfit(m, plan, d_obs).backward()
    rng = np.random.default_rng(0)
    dm = T.as_tensor(rng.standard_normal(m0.shape).astype(np.float32), device="cuda") * m0
    eps = 1e-3
    Jp = float(ag.fwi_misfit(m0 + eps * dm, plan, d_obs))
    Jm = float(ag.fwi_misfit(m0 - eps * dm, plan, d_obs))
    fd = (Jp - Jm) / (2 * eps)
    an = float((m.grad.double() * dm.double()).sum())
    assert fd == pytest.approx(an, rel=2e-3)


def test_forward_model_backward_is_the_adjoint(T, orc):
    from paper_2008_11778_gb300 import autograd as ag
    p, plan, d_obs = setup(T, orc)
    m = T.as_tensor(p.m_start.astype(np.float32), device="cuda").requires_grad_(True)
    d = ag.forward_model(m, plan)
    rng = np.random.default_rng(1)
    w = rng.standard_normal(plan.trace_count).astype(np.float32)
    (d * T.as_tensor(w, device="cuda")).sum().backward()
    m32 = p.m_start.astype(np.float32).astype(np.float64)
    ref = orc.born_adjoint(p.geom, m32, w) / m32
    assert rel(m.grad.cpu().numpy(), ref) < 1e-4


def test_born_backward_is_born_adjoint(T, orc):
    from paper_2008_11778_gb300 import autograd as ag
    p, plan, _ = setup(T, orc)
    m0 = T.as_tensor(p.m_true.astype(np.float32), device="cuda")
    rng = np.random.default_rng(2)
    rho = T.as_tensor(0.1 * rng.standard_normal(p.m_true.shape).astype(np.float32), device="cuda")
    rho.requires_grad_(True)
    w = rng.standard_normal(plan.trace_count).astype(np.float32)
    d = ag.born(rho, plan, m0)
    (d * T.as_tensor(w, device="cuda")).sum().backward()
    ref = orc.born_adjoint(p.geom, p.m_true.astype(np.float32), w)
    assert rel(rho.grad.cpu().numpy(), ref) < 1e-4
    # linearity: L(2 rho) = 2 L rho
    d2 = ag.born(2 * rho.detach(), plan, m0)
    assert rel(d2.cpu().numpy(), 2 * d.detach().cpu().numpy()) < 1e-6
