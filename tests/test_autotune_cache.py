"""Host logic of the autotuner's cache (no GPU): keys distinguish what the
launch configuration depends on, a stored tuning is reused, a different
device or geometry is tuned afresh, and a damaged cache file is ignored."""

from paper_2008_11778_gb300 import aafwi, synth


class FakeTuner:
    def __init__(self):
        self.calls = 0

    def __call__(self, geom, c_max, m, steps, reps, engine, max_workspace_bytes):
        self.calls += 1
        return {"engine": aafwi.ENGINE_PER_STEP, "tile_z": 64, "lanes": 0, "steps": steps,
                "table": [(1, 16, 4, 3.0), (1, 32, 4, 2.5), (1, 64, 4, 2.0)]}


def test_key_tracks_geometry_and_device():
    g = synth.tiny().geom
    k = aafwi.tune_key(g, 3000.0, "GB300", 152)
    assert k == aafwi.tune_key(synth.tiny().geom, 3000.0, "GB300", 152)
    assert k != aafwi.tune_key(g, 3000.0, "GB300", 148)
    assert k != aafwi.tune_key(g, 3000.0, "B200", 152)
    assert k != aafwi.tune_key(g, 3000.0, "GB300", 152, engine=aafwi.ENGINE_PER_STEP)
    g2 = synth.tiny().geom
    g2.nt = g2.nt.copy()
    g2.nt[0] -= 1
    assert k != aafwi.tune_key(g2, 3000.0, "GB300", 152)
    g3 = synth.tiny().geom
    g3.rec_ix = g3.rec_ix.copy()
    g3.rec_ix[0] = (g3.rec_ix[0] + 1) % g3.nx
    assert k != aafwi.tune_key(g3, 3000.0, "GB300", 152)


def test_cache_reuse_and_refresh(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    g = synth.tiny().geom
    t = FakeTuner()
    a = aafwi.autotune(g, 3000.0, None, cache_path=path, tuner=t, device=("GB300", 152))
    assert not a["cached"] and t.calls == 1 and a["tile_z"] == 64
    b = aafwi.autotune(g, 3000.0, None, cache_path=path, tuner=t, device=("GB300", 152))
    assert b["cached"] and t.calls == 1
    assert {k: v for k, v in b.items() if k != "cached"} == {k: v for k, v in a.items() if k != "cached"}
    c = aafwi.autotune(g, 3000.0, None, cache_path=path, tuner=t, device=("other", 100))
    assert not c["cached"] and t.calls == 2
    assert len(__import__("json").load(open(path))) == 2


def test_damaged_cache_is_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    t = FakeTuner()
    r = aafwi.autotune(synth.tiny().geom, 3000.0, None, cache_path=str(path), tuner=t, device=("GB300", 152))
    assert not r["cached"] and t.calls == 1
    assert aafwi.cache_lookup(str(path), aafwi.tune_key(synth.tiny().geom, 3000.0, "GB300", 152)) is not None
