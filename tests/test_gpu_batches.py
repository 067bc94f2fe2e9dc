"""Shot batches (plans whose wavefield buffers hold only some of the shots,
run one batch after another): bitwise the same traces, misfit, FWI and
LSRTM gradients and images as the plan that holds every shot, with the full
history and with checkpoints; the stored forward is not reusable."""
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
    p = synth.small_problem(nz=45, nx=150, nb=7, nt=140, S=5)
    g = p.geom
    g.nt = np.array([140, 97, 123, 140, 60], dtype=np.int32)
    return p


def run(A, plan, p, d_obs, rho, r):
    import torch
    m = torch.as_tensor(p.m_start.astype(np.float32), device="cuda")
    out = []
    d = torch.empty(plan.trace_count, device="cuda")
    plan.model_forward(m, d)
    out.append(d)
    g = torch.empty_like(m)
    out += [plan.adjoint_gradient(0, m, None, d_obs, g), g]
    db = torch.empty(plan.trace_count, device="cuda")
    out.append(plan.born_forward(m, rho, db))
    gl = torch.empty_like(m)
    out += [plan.adjoint_gradient(1, m, rho, d_obs, gl), gl]
    out.append(plan.born_adjoint(m, r, torch.empty_like(m)))
    out.append(plan.fwi_adjoint(m, r, torch.empty_like(m)))
    return out


@pytest.mark.parametrize("checkpoint_every", [1, 9], ids=["full", "checkpoints"])
@pytest.mark.parametrize("per_batch", [1, 2, 3])
def test_batches_bitwise_equal_to_one_batch(A, orc, checkpoint_every, per_batch):
    import torch
    p = ragged()
    g = p.geom
    d_obs = torch.as_tensor(orc.forward(g, p.m_true).astype(np.float32), device="cuda")
    rng = np.random.default_rng(3)
    rho = torch.as_tensor(rng.uniform(-0.1, 0.1, (g.nz, g.nx)).astype(np.float32), device="cuda")
    one = A.Plan(g, 3000.0, engine=A.ENGINE_PER_STEP, checkpoint_every=checkpoint_every)
    r = torch.as_tensor(rng.standard_normal(one.trace_count).astype(np.float32), device="cuda")
    bat = A.Plan(g, 3000.0, engine=A.ENGINE_PER_STEP, checkpoint_every=checkpoint_every, shots_per_batch=per_batch)
    assert one.info.n_batches == 1 and one.keeps_forward
    assert bat.info.shots_per_batch == per_batch and bat.info.n_batches == -(-5 // per_batch)
    assert not bat.keeps_forward
    ref = run(A, one, p, d_obs, rho, r)
    out = run(A, bat, p, d_obs, rho, r)
    for i, (a, b) in enumerate(zip(ref, out)):
        assert (torch.equal(a, b) if torch.is_tensor(a) else a == b), i


def test_batched_plan_refuses_forward_reuse_and_persistent_engine(A):
    import torch
    p = ragged()
    g = p.geom
    bat = A.Plan(g, 3000.0, shots_per_batch=2)
    assert bat.info.engine == A.ENGINE_PER_STEP
    m = torch.as_tensor(p.m_start.astype(np.float32), device="cuda")
    bat.model_forward(m)
    with pytest.raises(A.AafwiError) as e:
        bat.adjoint_gradient(0, m, None, torch.zeros(bat.trace_count, device="cuda"), torch.empty_like(m),
                             reuse_forward=True)
    assert e.value.code == 8
    with pytest.raises(A.AafwiError):
        A.Plan(g, 3000.0, shots_per_batch=2, engine=A.ENGINE_PERSISTENT)


def test_planner_checkpoints_then_batches_as_the_budget_shrinks(A):
    """On a grid too small to fill the GPU in batches, a budget below the
    full history gives checkpoints for all shots; a budget below that gives
    batches of shots with checkpoints; every plan stays within its budget."""
    p = ragged()
    g = p.geom
    one = A.Plan(g, 3000.0)
    assert one.info.checkpoint_every == 1 and one.info.n_batches == 1
    b1 = int(0.6 * one.info.workspace_bytes)
    ck = A.Plan(g, 3000.0, max_workspace_bytes=b1)
    assert ck.info.checkpoint_every > 1 and ck.info.n_batches == 1 and ck.info.workspace_bytes <= b1
    b2 = int(0.6 * ck.info.workspace_bytes)
    bat = A.Plan(g, 3000.0, max_workspace_bytes=b2)
    assert bat.info.checkpoint_every > 1 and bat.info.n_batches >= 2 and bat.info.workspace_bytes <= b2


def test_l2_sized_batches_of_the_lsrtm_workload(A):
    """l2_batches = 1 splits the LSRTM workload (64 shots of 280 x 777 padded
    cells) into even batches whose adjoint working set fits 40% of the L2 --
    4 batches of 16 on a GB300 -- and the LSRTM gradient stays bitwise that of
    the one-batch plan (records cut to 64 steps)."""
    import torch
    p = synth.lsrtm()
    g = p.geom.with_nt(64)
    one = A.Plan(g, 4700.0)
    split = A.Plan(g, 4700.0, l2_batches=1)
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    cap = max(1, int(0.4 * l2 / (3 * one.info.NZ * one.info.pitch * 4)))
    nb = -(-64 // cap)
    assert one.info.n_batches == 1
    assert split.info.n_batches == nb and split.info.shots_per_batch == -(-64 // nb)
    m0 = torch.as_tensor(p.m_true.astype(np.float32), device="cuda")
    rho = torch.as_tensor(p.extra["rho_true"].astype(np.float32), device="cuda")
    d = torch.empty(one.trace_count, device="cuda")
    one.born_forward(m0, rho, d)
    d2 = torch.empty_like(d)
    split.born_forward(m0, rho, d2)
    assert torch.equal(d, d2)
    g1, g2 = torch.empty_like(m0), torch.empty_like(m0)
    J1 = one.adjoint_gradient(A.MODE_LSRTM, m0, torch.zeros_like(rho), d, g1)
    J2 = split.adjoint_gradient(A.MODE_LSRTM, m0, torch.zeros_like(rho), d, g2)
    assert J1 == J2 and torch.equal(g1, g2)
    one.close()
    split.close()
