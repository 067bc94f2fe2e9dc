"""CUDA-graph replay of the per-step sweeps against launching them kernel by
kernel: bitwise equal traces, gradients and images (full history and
checkpoints, FWI and Born), the same kernel count per call, and a new
capture when the caller passes another buffer."""
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


def run_all(A, plan, p, d_obs, rho):
    """Every operator once; returns the outputs and the kernel launches of each call."""
    import torch
    m = torch.as_tensor(p.m_start.astype(np.float32), device="cuda")
    out, launches = {}, {}

    def counted(name, f):
        l0 = A.launch_count()
        out[name] = f()
        torch.cuda.synchronize()
        launches[name] = A.launch_count() - l0

    d = torch.empty(plan.trace_count, device="cuda")
    counted("forward", lambda: plan.model_forward(m, d).clone())
    g = torch.empty_like(m)
    counted("fwi", lambda: (plan.adjoint_gradient(0, m, None, d_obs, g), g.clone()))
    db = torch.empty(plan.trace_count, device="cuda")
    counted("born", lambda: plan.born_forward(m, rho, db).clone())
    gl = torch.empty_like(m)
    counted("lsrtm", lambda: (plan.adjoint_gradient(1, m, rho, d_obs, gl), gl.clone()))
    im = torch.empty_like(m)
    counted("rtm", lambda: plan.born_adjoint(m, d_obs, im).clone())
    return out, launches


@pytest.mark.parametrize("checkpoint_every", [1, 7], ids=["full", "checkpoints"])
def test_graph_replay_equals_kernel_by_kernel(A, orc, checkpoint_every):
    import torch
    p = synth.tiny()
    g = p.geom
    d_obs = torch.as_tensor(orc.forward(g, p.m_true).astype(np.float32), device="cuda")
    rho = torch.as_tensor(np.random.default_rng(5).uniform(-0.1, 0.1, (g.nz, g.nx)).astype(np.float32),
                          device="cuda")
    plain = A.Plan(g, 3000.0, engine=A.ENGINE_PER_STEP, checkpoint_every=checkpoint_every, graphs=False)
    graph = A.Plan(g, 3000.0, engine=A.ENGINE_PER_STEP, checkpoint_every=checkpoint_every, graphs=True)
    o1, l1 = run_all(A, plain, p, d_obs, rho)
    o2, l2 = run_all(A, graph, p, d_obs, rho)          # first calls: capture, then replay
    o3, l3 = run_all(A, graph, p, d_obs, rho)          # cached graphs (new caller buffers: re-capture)
    for k in o1:
        a, b, c = o1[k], o2[k], o3[k]
        if isinstance(a, tuple):
            assert a[0] == b[0] == c[0], k
            a, b, c = a[1], b[1], c[1]
        assert torch.equal(a, b) and torch.equal(a, c), k
    assert l1 == l2 == l3


def test_graph_cache_reuses_and_recaptures(A):
    """born_forward writes the caller's trace buffer from inside the sweep, so
    each new buffer is a new capture; a buffer seen before replays its graph."""
    import torch
    p = synth.tiny()
    g = p.geom
    plan = A.Plan(g, 3000.0, engine=A.ENGINE_PER_STEP, graphs=True)
    m = torch.as_tensor(p.m_start.astype(np.float32), device="cuda")
    rho = torch.full_like(m, 0.05)
    outs = [torch.empty(plan.trace_count, device="cuda") for _ in range(3)]
    plan.born_forward(m, rho, outs[0])
    for d in outs[1:] + outs[:1]:                       # new buffers, then the first again
        d.fill_(float("nan"))
        plan.born_forward(m, rho, d)
    torch.cuda.synchronize()
    for d in outs[1:]:
        assert torch.equal(d, outs[0])
    assert torch.isfinite(outs[0]).all() and outs[0].abs().max() > 0


@pytest.mark.parametrize("checkpoint_every", [1, 7], ids=["full", "checkpoints"])
@pytest.mark.parametrize("graphs", [False, True], ids=["launches", "graphs"])
def test_dependent_launches_equal_plain_launches(A, orc, checkpoint_every, graphs):
    """Programmatic dependent launches (each step kernel resident while the
    previous one drains, the adjoint's T^n copy issued before the grid wait)
    give bitwise the results of plain launches, with the same launch count;
    the records are uneven, so in the one-shot batches of the third plan
    whole launches have no active CTA."""
    import torch
    p = synth.tiny()
    g = p.geom
    g.nt = np.array([600, 410, 520], dtype=np.int32)
    d_obs = torch.as_tensor(orc.forward(g, p.m_true).astype(np.float32), device="cuda")
    rho = torch.as_tensor(np.random.default_rng(6).uniform(-0.1, 0.1, (g.nz, g.nx)).astype(np.float32),
                          device="cuda")
    kw = dict(engine=A.ENGINE_PER_STEP, checkpoint_every=checkpoint_every, graphs=graphs)
    o1, l1 = run_all(A, A.Plan(g, 3000.0, pdl=False, **kw), p, d_obs, rho)
    o2, l2 = run_all(A, A.Plan(g, 3000.0, pdl=True, **kw), p, d_obs, rho)
    o3, l3 = run_all(A, A.Plan(g, 3000.0, pdl=True, shots_per_batch=1, **kw), p, d_obs, rho)
    for k in o1:
        a, b, c = o1[k], o2[k], o3[k]
        if isinstance(a, tuple):
            assert a[0] == b[0] == c[0], k
            a, b, c = a[1], b[1], c[1]
        assert torch.equal(a, b) and torch.equal(a, c), k
    assert l1 == l2


@pytest.mark.parametrize("nt", [[600, 600, 600], [599, 410, 523]], ids=["even", "odd-uneven"])
@pytest.mark.parametrize("spb", [0, 1], ids=["one-batch", "one-shot-batches"])
def test_two_step_forward_equals_one_step(A, orc, nt, spb):
    """The two-step forward kernel (tile + 4-cell ring advanced to n+1 in
    shared memory, then the tile to n+2) gives bitwise the traces, the stored
    T^n (through the FWI gradient) and the misfit of one step per launch;
    odd record lengths end with a one-step launch, shots whose record ends
    after the first of a launch's two steps stop there."""
    import torch
    p = synth.tiny()
    g = p.geom
    g.nt = np.array(nt, dtype=np.int32)
    d_obs = torch.as_tensor(orc.forward(g, p.m_true).astype(np.float32), device="cuda")
    rho = torch.as_tensor(np.random.default_rng(7).uniform(-0.1, 0.1, (g.nz, g.nx)).astype(np.float32),
                          device="cuda")
    one = A.Plan(g, 3000.0, engine=A.ENGINE_PER_STEP, steps_per_launch=1, shots_per_batch=spb)
    two = A.Plan(g, 3000.0, engine=A.ENGINE_PER_STEP, steps_per_launch=2, shots_per_batch=spb)
    assert one.info.steps_per_launch == 1 and two.info.steps_per_launch == 2
    o1, l1 = run_all(A, one, p, d_obs, rho)
    o2, l2 = run_all(A, two, p, d_obs, rho)
    for k in o1:
        a, b = o1[k], o2[k]
        if isinstance(a, tuple):
            assert a[0] == b[0], k
            a, b = a[1], b[1]
        assert torch.equal(a, b), k
    nb, lanes = two.info.n_batches, two.info.lanes
    assert l2["forward"] == l1["forward"] - nb * lanes * (max(nt) // 2)


@pytest.mark.parametrize("graphs", [False, True], ids=["launches", "graphs"])
@pytest.mark.parametrize("checkpoint_every", [1, 7], ids=["full", "checkpoints"])
def test_shot_lanes_equal_one_lane(A, orc, graphs, checkpoint_every):
    """Shot lanes (the batch's shots in groups whose launch chains run on
    forked streams) give bitwise the results of one chain, for every
    operator, uneven records included."""
    import torch
    p = synth.small_problem(nz=40, nx=70, nb=10, nt=200, S=5)
    g = p.geom
    g.nt = np.array([200, 131, 200, 77, 163], dtype=np.int32)
    d_obs = torch.as_tensor(orc.forward(g, p.m_true).astype(np.float32), device="cuda")
    rho = torch.as_tensor(np.random.default_rng(8).uniform(-0.1, 0.1, (g.nz, g.nx)).astype(np.float32),
                          device="cuda")
    kw = dict(engine=A.ENGINE_PER_STEP, checkpoint_every=checkpoint_every, graphs=graphs)
    outs = []
    for lanes in (1, 2, 4):
        plan = A.Plan(g, 3000.0, lanes=lanes, **kw)
        assert plan.info.lanes == lanes
        outs.append(run_all(A, plan, p, d_obs, rho))
    (o1, l1) = outs[0]
    for o, l in outs[1:]:
        for k in o1:
            a, b = o1[k], o[k]
            if isinstance(a, tuple):
                assert a[0] == b[0], k
                a, b = a[1], b[1]
            assert torch.equal(a, b), k
