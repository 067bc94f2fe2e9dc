"""Write the stored expected values under tests/golden/ from the FP64 oracle.

Calls only oracle/ (and the seeded input generators); nothing here comes from
the CUDA library.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle                                   # noqa: E402
from oracle import aa                           # noqa: E402
from paper_2008_11778_gb300 import synth        # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

# Fixed step of eq. GD: eta = ETA_FACTOR * max|p_0| / max|grad J(p_0)|.  The
# cells next to the sources dominate the Hessian; with this factor plain
# steepest descent is stable on the tiny problem (it diverges at 3e-4).
ETA_FACTOR = 1e-4


def tiny_aa_history():
    """Alg. 2 on the tiny two-layer problem: AA(5), fixed eta, 10 iterations.

    eta = ETA_FACTOR ||p_0||_inf / ||grad J(p_0)||_inf (the step-size reading), the
    unknown p = m = 1/c^2 clipped to the velocity bounds after each update.
    """
    p = synth.tiny()
    g = p.geom
    d_obs = oracle.forward(g, p.m_true)
    J0, g0 = oracle.fwi_gradient(g, p.m_start, d_obs)
    eta = ETA_FACTOR * np.abs(p.m_start).max() / np.abs(g0).max()
    out = aa.aa_gd(lambda m: oracle.fwi_gradient(g, m, d_obs),
                   p.m_start, M=p.M, eta=eta, iters=p.iters, bounds=p.m_bounds,
                   misfit_fn=lambda m: 0.5 * float(np.sum((oracle.forward(g, m) - d_obs) ** 2)))
    sd = aa.aa_gd(lambda m: oracle.fwi_gradient(g, m, d_obs),
                  p.m_start, M=0, eta=eta, iters=p.iters, bounds=p.m_bounds)
    return {
        "what": "FP64 oracle, Alg. 2 (AA(5) on steepest descent, fixed eta, Armijo "
                "backtracking lambda in 1,1/2,1/4,1/8), tiny two-layer problem "
                "101x51, 3 shots, 600 steps; J[k] = J(p_k), k = 0..10",
        "eta_factor": ETA_FACTOR,
        "eta": float(eta),
        "J": [float(x) for x in out["J"]],
        "lam": [float(x) for x in out["lam"]],
        "Mk": [int(x) for x in out["Mk"]],
        "n_trials": int(out["n_trials"]),
        "J_sd": [float(x) for x in sd["J"]],
    }


if __name__ == "__main__":
    res = tiny_aa_history()
    with open(os.path.join(HERE, "tiny_aa_history.json"), "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res, indent=1))
