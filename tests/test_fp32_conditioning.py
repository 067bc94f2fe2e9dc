"""Why the tiny problem's 10-iteration misfit history cannot match the FP64
oracle to 1e-3 with FP32 wavefields (CPU only, explains a tolerance).

An FP32 forward (float32 numpy emulation of the kernel's evaluation order) is
combined with the oracle's exact FP64 adjoint and Anderson iteration.  Its
traces agree with the FP64 recurrence to ~1e-6, within the 1e-5 seismogram
target, yet the Alg. 2 misfit history departs by more than 1e-3 within a few
iterations: the residual is ~0.2 % of the data and the AA extrapolation
amplifies the remaining difference.  The same order of departure is accepted
for the GPU history in tests/test_gpu_parity.py.
"""
import json
import os

import numpy as np
import pytest

from paper_2008_11778_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.slow
def test_fp32_forward_alone_moves_the_tiny_aa_history(orc):
    from oracle import aa
    from fp32_emulation import forward_fp32
    with open(os.path.join(HERE, "golden", "tiny_aa_history.json")) as f:
        ref = json.load(f)
    p = synth.tiny()
    g = p.geom
    d_obs = orc.forward(g, p.m_true).astype(np.float32).astype(np.float64)
    m32 = p.m_start.astype(np.float32)
    d32 = forward_fp32(g, m32)
    d64 = orc.forward(g, m32)
    trace_err = np.linalg.norm(d32 - d64) / np.linalg.norm(d64)
    resid_ratio = np.linalg.norm(d64 - d_obs) / np.linalg.norm(d_obs)
    assert trace_err < 1e-5 and resid_ratio < 5e-3

    def grad_fn(m):
        mm = m.astype(np.float32)
        r = forward_fp32(g, mm) - d_obs
        return 0.5 * float(r @ r), orc.born_adjoint(g, mm.astype(np.float64), r) / mm.astype(np.float64)

    def misfit(m):
        r = forward_fp32(g, m.astype(np.float32)) - d_obs
        return 0.5 * float(r @ r)

    iters = 6
    out = aa.aa_gd(grad_fn, p.m_start, M=5, eta=ref["eta"], iters=iters, bounds=p.m_bounds,
                   misfit_fn=misfit)
    J, Jr = np.array(out["J"]), np.array(ref["J"][:iters + 1])
    dev_early = np.linalg.norm(J[:4] - Jr[:4]) / np.linalg.norm(Jr[:4])
    dev_all = np.linalg.norm(J - Jr) / np.linalg.norm(Jr)
    assert dev_early < 1e-3          # before the AA extrapolation takes over
    assert dev_all > 1e-3            # FP32 wavefields alone exceed the 1e-3 history target


@pytest.mark.slow
def test_accumulation_order_of_the_stencil(orc):
    """The kernels add the four weighted differences from the smallest weight
    up, so the dominant 8064 d1 term enters unrounded through the last fma.
    On the tiny problem's start model that order's FP32 traces are closer to
    the FP64 recurrence than the largest-first or plain orders, and within
    1.5e-6 of it."""
    from fp32_emulation import forward_fp32
    p = synth.tiny()
    g = p.geom
    m32 = p.m_start.astype(np.float32)
    d64 = orc.forward(g, m32)
    err = {o: np.linalg.norm(forward_fp32(g, m32, order=o) - d64) / np.linalg.norm(d64)
           for o in ("small_first", "large_first", "plain")}
    assert err["small_first"] < err["large_first"] and err["small_first"] < err["plain"]
    assert err["small_first"] < 1.5e-6
