"""The committed learned-vs-plain evaluation record
(paper_2008_11778_gb300/weights/unet_c32_eval.json) is internally consistent:
its summary is exactly what `learned.summarize` computes from its per-model
rows, and the per-model arrays agree with the rows (no GPU needed)."""
import json

import numpy as np


def _record():
    from paper_2008_11778_gb300 import learned
    with open(learned.EVAL_RECORD) as f:
        return json.load(f)


def test_record_summary_recomputes_from_its_rows():
    from paper_2008_11778_gb300 import learned
    rec = _record()
    s = rec["summary"]
    again = learned.summarize(rec["rows"], s["target"], s["max_iters"])
    assert again == s


def test_record_rows_and_flags_agree():
    rec = _record()
    s, rows = rec["summary"], rec["rows"]
    assert s["models"] == len(rows) == 50
    assert s["learned_reached"] == sum(r["learned"]["reached"] for r in rows)
    assert s["plain_reached"] == sum(r["plain"]["reached"] for r in rows)
    # a run that reached the target ends at or below it; one that did not used every iteration
    for r in rows:
        for arm in [r["learned"], r["plain"], *r["plain_eta"].values()]:
            if arm["reached"]:
                assert arm["J_over_J0"] <= s["target"]
            else:
                assert arm["iterations"] >= s["max_iters"]
    sp = np.array(s["plain_s"]) / np.array(s["learned_s"])
    assert abs(float(np.median(sp)) - s["median_speedup"]) < 1e-12
