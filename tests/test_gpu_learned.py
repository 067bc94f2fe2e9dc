"""The trained learned preconditioner (weights committed under
paper_2008_11778_gb300/weights, produced by `python -m
paper_2008_11778_gb300.learned`) against plain AA(10) on a held-out
400 x 150 model: wall seconds and iterations to J/J0 <= 1e-2 on the same GPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    from paper_2008_11778_gb300 import aafwi, build, learned
    build.build()
    aafwi.load()
    assert torch.cuda.is_available()
    return aafwi, learned


def test_learned_step_features_and_apply(mods):
    import torch
    aafwi, learned = mods
    rng = np.random.default_rng(0)
    g = torch.as_tensor(rng.standard_normal((5, 7)).astype(np.float32), device="cuda")
    m = torch.as_tensor(rng.uniform(1, 2, (5, 7)).astype(np.float32), device="cuda")
    x = torch.full((2, 8, 8), 7.0, device="cuda")
    st = torch.empty(3, dtype=torch.float64, device="cuda")
    aafwi.learned_features(g, m, 8, 8, x, st)
    gh, mh = g.cpu().numpy().astype(np.float64), m.cpu().numpy().astype(np.float64)
    s = st.cpu().numpy()
    assert s[0] == pytest.approx(np.abs(gh).max()) and s[1] == pytest.approx(mh.mean())
    assert s[2] == pytest.approx(mh.std(), rel=1e-6)
    xh = x.cpu().numpy()
    np.testing.assert_allclose(xh[0, :5, :7], gh / s[0], rtol=1e-6)
    np.testing.assert_allclose(xh[1, :5, :7], (mh - s[1]) / s[2], rtol=1e-5, atol=1e-6)
    assert (xh[:, 5:, :] == 0).all() and (xh[:, :, 7:] == 0).all()
    d = torch.as_tensor(rng.standard_normal((8, 8)).astype(np.float32), device="cuda")
    out = torch.empty_like(m)
    aafwi.learned_apply(m, d, st, out, 1.2, 1.8)
    ref = np.clip(mh + s[2] * d.cpu().numpy()[:5, :7], 1.2, 1.8)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-6)


@pytest.mark.slow
def test_learned_aa_beats_plain_aa_on_held_out_model(mods):
    aafwi, learned = mods
    params, meta = learned.load_weights()
    rows = learned.compare(params, n_eval=1, target=1e-2, max_iters=120, log=lambda *a: None)
    r = rows[0]
    assert r["learned"]["reached"]
    assert r["learned"]["learned_steps"] >= 1
    assert r["learned"]["iterations"] < r["plain"]["iterations"]
    assert r["learned"]["seconds"] < r["plain"]["seconds"]
