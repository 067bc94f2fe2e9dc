"""Tile heights of the per-step kernels and the autotuner: every tile gives
bitwise the same traces and gradient; the tuner times each qualifying
configuration, returns the fastest, and a plan built from its (cached)
choice matches a plan built with those options by hand."""
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


def outputs(A, plan, p, d_obs):
    import torch
    m = torch.as_tensor(p.m_start.astype(np.float32), device="cuda")
    d = torch.empty(plan.trace_count, device="cuda")
    plan.model_forward(m, d)
    g = torch.empty_like(m)
    J = plan.adjoint_gradient(0, m, None, d_obs, g)
    return d, J, g


def test_tile_heights_bitwise_equal(A, orc):
    import torch
    p = synth.small_problem(nz=70, nx=150, nb=9, nt=150, S=3)   # 88 padded rows: ragged for all tiles
    g = p.geom
    d_obs = torch.as_tensor(orc.forward(g, p.m_true).astype(np.float32), device="cuda")
    ref = None
    for tz in (16, 32, 64):
        plan = A.Plan(g, 3000.0, engine=A.ENGINE_PER_STEP, tile_z=tz)
        assert plan.info.tile_z == tz
        out = outputs(A, plan, p, d_obs)
        if ref is None:
            ref = out
        else:
            assert torch.equal(out[0], ref[0]) and out[1] == ref[1] and torch.equal(out[2], ref[2]), tz
    with pytest.raises(A.AafwiError):
        A.Plan(g, 3000.0, tile_z=24)


def test_autotune_picks_the_fastest_and_plans_follow_it(A, orc, tmp_path):
    import torch
    p = synth.tiny()
    g = p.geom
    m = torch.as_tensor(p.m_start.astype(np.float32), device="cuda")
    res = A.run_autotune(g, 3000.0, m, steps=40, reps=2)
    kinds = {(e, t) for e, t, _, _ in res["table"]}
    assert {(A.ENGINE_PER_STEP, 16), (A.ENGINE_PER_STEP, 32), (A.ENGINE_PER_STEP, 64)} <= kinds
    assert (A.ENGINE_PERSISTENT, 0) in kinds                      # the tiny plan keeps its full history
    assert {(A.ENGINE_HYBRID, 16), (A.ENGINE_HYBRID, 32), (A.ENGINE_HYBRID, 64)} <= kinds
    assert all(ms > 0 for _, _, _, ms in res["table"])
    best = min(res["table"], key=lambda e: e[3])
    assert (res["engine"], res["tile_z"]) == (best[0], best[1])
    assert res["lanes"] in (0, best[2])                  # 0: the default lanes won
    if res["engine"] != A.ENGINE_PERSISTENT:            # the winner re-timed with 1 and 2 lanes (3 shots)
        assert {l for e, t, l, _ in res["table"] if (e, t) == (res["engine"], res["tile_z"])} >= {1, 2, 3}
    only = A.run_autotune(g, 3000.0, m, steps=40, reps=1, engine=A.ENGINE_PER_STEP)
    assert {e for e, _, _, _ in only["table"]} == {A.ENGINE_PER_STEP}

    cache = str(tmp_path / "tune.json")
    tuned = A.Plan(g, 3000.0, tune_model=m, tune_cache=cache)
    again = A.Plan(g, 3000.0, tune_model=m, tune_cache=cache)
    assert not tuned.tuning["cached"] and again.tuning["cached"]
    assert (again.info.engine, again.tuning["tile_z"]) == (tuned.info.engine, tuned.tuning["tile_z"])
    assert again.info.lanes == tuned.info.lanes
    manual = A.Plan(g, 3000.0, engine=tuned.tuning["engine"], tile_z=tuned.tuning["tile_z"])
    d_obs = torch.as_tensor(orc.forward(g, p.m_true).astype(np.float32), device="cuda")
    a, b = outputs(A, tuned, p, d_obs), outputs(A, manual, p, d_obs)
    assert torch.equal(a[0], b[0]) and a[1] == b[1] and torch.equal(a[2], b[2])


def test_autotune_reports_a_bad_model(A):
    import torch
    p = synth.tiny()
    m = torch.full((p.geom.nz, p.geom.nx), float("nan"), device="cuda")
    with pytest.raises(A.AafwiError) as e:
        A.run_autotune(p.geom, 3000.0, m, steps=8, reps=1)
    assert e.value.code == 4
