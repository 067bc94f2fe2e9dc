"""The persistent engine (one cooperative launch per sweep, strips of rows in
shared memory) against the one-launch-per-step engine: bitwise equal traces,
gradients and images, and a bounded wait that reports a timeout."""
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


def ragged():
    p = synth.small_problem(nz=45, nx=150, nb=7, nt=140, S=3)
    g = p.geom
    g.nt = np.array([140, 97, 123], dtype=np.int32)
    g.rec_off = np.array([0, 30, 30, 95], dtype=np.int32)
    rng = np.random.default_rng(0)
    g.rec_iz = rng.integers(0, g.nz, 95).astype(np.int32)
    g.rec_ix = np.concatenate([rng.choice(g.nx, 30, replace=False),
                               rng.choice(g.nx, 65, replace=False)]).astype(np.int32)
    g.src_iz = np.array([0, 20, 44], dtype=np.int32)
    g.src_ix = np.array([0, 77, 149], dtype=np.int32)
    return p


@pytest.mark.parametrize("make", [synth.tiny, ragged], ids=["tiny", "ragged"])
def test_persistent_equals_per_step_bitwise(A, orc, make):
    import torch
    p = make()
    g = p.geom
    c_max = 3000.0
    per = A.Plan(g, c_max, engine=A.ENGINE_PER_STEP)
    pst = A.Plan(g, c_max, engine=A.ENGINE_PERSISTENT)
    hyb = A.Plan(g, c_max, engine=A.ENGINE_HYBRID)
    assert per.info.engine == A.ENGINE_PER_STEP and pst.info.engine == A.ENGINE_PERSISTENT
    assert hyb.info.engine == A.ENGINE_HYBRID
    m = torch.as_tensor(p.m_start.astype(np.float32), device="cuda")
    d_obs = torch.as_tensor(orc.forward(g, p.m_true).astype(np.float32), device="cuda")
    r = torch.as_tensor(np.random.default_rng(1).standard_normal(per.trace_count).astype(np.float32),
                        device="cuda")
    rho = torch.as_tensor(np.random.default_rng(2).uniform(-0.1, 0.1, (g.nz, g.nx)).astype(np.float32),
                          device="cuda")

    def run(plan):
        d = torch.empty(plan.trace_count, device="cuda")
        plan.model_forward(m, d)
        gr, im, gl = torch.empty_like(m), torch.empty_like(m), torch.empty_like(m)
        J = plan.adjoint_gradient(0, m, None, d_obs, gr)
        plan.born_adjoint(m, r, im)
        Jl = plan.adjoint_gradient(1, m, rho, d_obs, gl)      # Born forward per step, adjoint per engine
        return d, J, gr, im, Jl, gl

    ref = run(per)
    for plan in (pst, hyb):
        out = run(plan)
        for a, b in zip(ref, out):
            assert (torch.equal(a, b) if torch.is_tensor(a) else a == b)


def test_batched_plan_qualifies_for_the_persistent_engine(A):
    p = synth.batched()
    plan = A.Plan(p.geom, c_max=p.c_bounds[1], engine=A.ENGINE_PERSISTENT)
    assert plan.info.engine == A.ENGINE_PERSISTENT
    assert plan.info.persist_ctas >= 100
    assert plan.info.checkpoint_every == 1
    auto = A.Plan(p.geom, c_max=p.c_bounds[1])
    assert auto.info.engine == A.ENGINE_PER_STEP and auto.info.tile_z == 16


def test_bounded_wait_reports_timeout_and_context_survives(A, orc):
    import torch
    p = synth.small_problem(nz=40, nx=70, nb=10, nt=120, S=2)
    plan = A.Plan(p.geom, 3000.0, engine=A.ENGINE_PERSISTENT)
    m = torch.as_tensor(p.m_start.astype(np.float32), device="cuda")
    d_obs = torch.zeros(plan.trace_count, device="cuda")
    grad = torch.empty_like(m)
    plan.set_stall(10)
    with pytest.raises(A.AafwiError) as e:
        plan.adjoint_gradient(0, m, None, d_obs, grad)
    assert e.value.code == 5                       # TIMEOUT
    plan.set_stall(-1)
    J = plan.adjoint_gradient(0, m, None, d_obs, grad)
    assert np.isfinite(J) and torch.isfinite(grad).all()
    per = A.Plan(p.geom, 3000.0, engine=A.ENGINE_PER_STEP)
    g2 = torch.empty_like(m)
    assert per.adjoint_gradient(0, m, None, d_obs, g2) == J and torch.equal(grad, g2)
