"""The LSRTM (737 x 240, 64 shots, 4000 steps) and large (2001 x 601, 200
shots, 6000 steps) workloads at full grid size: outputs the FP64 oracle can
compute one shot at a time, and properties that hold at any size on the
plans the planner builds for all shots (shot batches)."""
import numpy as np
import pytest

from paper_2008_11778_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TRACE_TOL = 1e-5
GRAD_TOL = 1e-4


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_2008_11778_gb300 import aafwi, build
    build.build()
    aafwi.load()
    assert torch.cuda.is_available()
    return torch, aafwi


def dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def test_lsrtm_one_shot_born_traces_and_gradient(gpu, orc):
    """One shot of the LSRTM geometry at full size and record length: Born
    traces and the LSRTM gradient against the oracle."""
    torch, A = gpu
    p = synth.lsrtm()
    g = p.geom.subset([len(p.geom.src_iz) // 2])
    m0 = p.m_true.astype(np.float32)
    rho_true = p.extra["rho_true"].astype(np.float32)
    plan = A.Plan(g, 4700.0)
    d = torch.empty(plan.trace_count, device="cuda")
    plan.born_forward(dev(torch, m0), dev(torch, rho_true), d)
    ref = orc.born_forward(g, m0, rho_true)
    assert rel(host(d), ref) < TRACE_TOL
    rho = (0.5 * rho_true).astype(np.float32)
    d_obs = ref.astype(np.float32)
    J_ref, g_ref = orc.lsrtm_gradient(g, m0, rho, d_obs)
    grad = torch.empty(m0.shape, device="cuda")
    J = plan.adjoint_gradient(1, dev(torch, m0), dev(torch, rho), dev(torch, d_obs), grad)
    assert abs(J - J_ref) / J_ref < 1e-4
    assert rel(host(grad), g_ref) < GRAD_TOL


def test_lsrtm_all_shots_dot_product(gpu):
    """<L rho, d> = <rho, L^T d> on the plan of all 64 shots (the exact
    discrete adjoint: only FP32 rounding separates the two sides)."""
    torch, A = gpu
    p = synth.lsrtm()
    g = p.geom
    plan = A.Plan(g, 4700.0)
    rng = np.random.default_rng(11)
    m0 = dev(torch, p.m_true)
    rho = dev(torch, rng.standard_normal((g.nz, g.nx)))
    d = dev(torch, rng.standard_normal(plan.trace_count))
    Lr = torch.empty(plan.trace_count, device="cuda")
    plan.born_forward(m0, rho, Lr)
    Ltd = torch.empty_like(m0)
    plan.born_adjoint(m0, d, Ltd)
    a = float(torch.dot(Lr.double(), d.double()))
    b = float(torch.dot(rho.double().ravel(), Ltd.double().ravel()))
    assert abs(a - b) / max(abs(a), abs(b)) < 1e-4


def test_large_grid_one_shot_traces(gpu, orc):
    """The 2001 x 601 grid (pitch 2048 floats, 16 tiles across) with the
    widest spread of the large workload, record cut to 1500 steps so that
    the oracle stays within seconds: traces against the oracle."""
    torch, A = gpu
    p = synth.large()
    g0 = p.geom
    s = int(np.argmax(g0.nrec))
    g = g0.subset([s]).with_nt(1500)
    m = p.m_start.astype(np.float32)
    plan = A.Plan(g, p.c_bounds[1])
    d = torch.empty(plan.trace_count, device="cuda")
    plan.model_forward(dev(torch, m), d)
    assert rel(host(d), orc.forward(g, m)) < TRACE_TOL


def test_large_all_shots_planner_and_batches(gpu):
    """All 200 shots of the large workload: the planner splits them into
    batches; the batched plan's traces of a shot are bitwise those of a
    one-shot plan, and its FWI gradient is finite and nonzero."""
    torch, A = gpu
    p = synth.large()
    g = p.geom.with_nt(600)          # full grid and all shots; record cut to keep the test short
    plan = A.Plan(g, p.c_bounds[1], max_workspace_bytes=24 << 30)
    assert plan.info.n_batches > 1
    m = dev(torch, p.m_start)
    d = torch.empty(plan.trace_count, device="cuda")
    plan.model_forward(m, d)
    off = g.trace_offsets()
    for s in (0, 117, 199):
        one = A.Plan(g.subset([s]), p.c_bounds[1])
        ds = torch.empty(one.trace_count, device="cuda")
        one.model_forward(m, ds)
        assert torch.equal(ds, d[off[s]:off[s + 1]]), s
        del one
    d_obs = d * 1.01
    grad = torch.empty_like(m)
    J = plan.adjoint_gradient(0, m, None, d_obs, grad)
    assert J > 0 and torch.isfinite(grad).all() and grad.abs().max() > 0


def test_large_gradient_in_the_benchmarks_launch_configuration(gpu, orc):
    """The large grid in the launch configuration the benchmark times: the
    planner's L2-sized batches (6 shots spread over the line -> 2 batches of
    3 on a GB300), two lanes, 16-row tiles, records cut to 600 steps.  With
    zero observed data the residual is the data itself (every receiver sees
    the direct wave), so J and the FWI gradient meet the 1e-4 target against
    the oracle."""
    torch, A = gpu
    p = synth.large()
    g = p.geom.subset([0, 40, 80, 120, 160, 199]).with_nt(600)
    plan = A.Plan(g, p.c_bounds[1], engine=A.ENGINE_PER_STEP, tile_z=16, lanes=2, l2_batches=1)
    assert plan.info.n_batches == 2 and plan.info.shots_per_batch == 3 and plan.info.lanes == 2
    m = p.m_start.astype(np.float32)
    d_obs = np.zeros(g.trace_count(), dtype=np.float32)
    J_ref, g_ref = orc.fwi_gradient(g, m, d_obs)
    grad = torch.empty(m.shape, device="cuda")
    J = plan.adjoint_gradient(0, dev(torch, m), None, dev(torch, d_obs), grad)
    assert abs(J - J_ref) / J_ref < 1e-4
    assert rel(host(grad), g_ref) < GRAD_TOL
    plan.close()
