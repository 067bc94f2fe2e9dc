"""The stored expected values under tests/golden/ are what the oracle computes.

tiny_aa_history.json is written by tests/golden/make_golden.py (oracle only);
this test recomputes it so that a stale file cannot pass as a target.
"""
import json
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.slow
def test_tiny_aa_history_is_current(orc):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(HERE, "tiny_aa_history.json")) as f:
        stored = json.load(f)
    now = mg.tiny_aa_history()
    np.testing.assert_allclose(now["J"], stored["J"], rtol=1e-9)
    assert now["lam"] == stored["lam"] and now["Mk"] == stored["Mk"]
    # Alg. 2 accelerates plain steepest descent at the same fixed step
    assert stored["J"][-1] < 0.75 * stored["J_sd"][-1]
    assert all(b <= a for a, b in zip(stored["J"][1:], stored["J"][2:]))
