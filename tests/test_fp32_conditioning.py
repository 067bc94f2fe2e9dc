"""The FP32 floor of the tiny problem's end-to-end parity (CPU only).

The tiny problem's stated targets are a gradient within 1e-4 and a
10-iteration Alg. 2 misfit history within 1e-3 of the FP64 oracle.  Its
residual is only ~0.1 % of the data, so a forward trace error e (relative to
the data) is ~1000 e relative to the residual, and the gradient is linear in
the residual.  These tests measure, with a float32 emulation of the
recurrence (tests/fp32_emulation.py) combined with the oracle's exact FP64
adjoint and Anderson iteration, how close FP32 wavefields can come:

  form          traces    gradient   history (10 it.)
  kernel        1.1e-6    1.3e-3     2.3e-2     (the library's kernels)
  increment     2.1e-7    3.1e-4     1.6e-2     (u, v = u^n - u^{n-1})
  compensated   9.9e-8    2.0e-4     1.6e-2     (u as an FP32 pair)
  double_uv     8.0e-8    --         --         (u and v as FP32 pairs)

The FP32 stencil itself sets the last floor: with both state fields carried
in pairs the traces stay at 8e-8.  The history departs through the AA
extrapolation, which amplifies errors that are correlated with the model:
random data perturbations of 1e-7 move the oracle's own history by only
~2e-5.  So neither target of the tiny problem is met by FP32 wavefields;
the GPU tests record them as unmet (strict xfail) and bound the measured
departure.  The adjoint operator, and problems whose residual is the size of
the data, meet the targets.
"""
import json
import os

import numpy as np
import pytest

from paper_2008_11778_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _fp32_aa(orc, form, iters):
    from oracle import aa
    from fp32_emulation import forward_fp32
    with open(os.path.join(HERE, "golden", "tiny_aa_history.json")) as f:
        ref = json.load(f)
    p = synth.tiny()
    g = p.geom
    d_obs = orc.forward(g, p.m_true).astype(np.float32).astype(np.float64)

    def grad_fn(m):
        mm = m.astype(np.float32)
        r = forward_fp32(g, mm, form=form) - d_obs
        return 0.5 * float(r @ r), orc.born_adjoint(g, mm.astype(np.float64), r) / mm.astype(np.float64)

    def misfit(m):
        r = forward_fp32(g, m.astype(np.float32), form=form) - d_obs
        return 0.5 * float(r @ r)

    m32 = p.m_start.astype(np.float32).astype(np.float64)
    _, g_ref = orc.fwi_gradient(g, m32, d_obs)
    _, g_emu = grad_fn(p.m_start)
    out = aa.aa_gd(grad_fn, p.m_start, M=5, eta=ref["eta"], iters=iters, bounds=p.m_bounds,
                   misfit_fn=misfit)
    J, Jr = np.array(out["J"]), np.array(ref["J"][:iters + 1])
    return (np.linalg.norm(g_emu - g_ref) / np.linalg.norm(g_ref),
            np.linalg.norm(J - Jr) / np.linalg.norm(Jr), np.linalg.norm(J[:4] - Jr[:4]) / np.linalg.norm(Jr[:4]))


@pytest.mark.slow
def test_kernel_form_floor_of_the_tiny_gradient_and_history(orc):
    """The kernels' FP32 form: traces within the 1e-5 seismogram target, the
    gradient at ~1e-3 and the 10-iteration history at ~2e-2 of the oracle."""
    from fp32_emulation import forward_fp32
    p = synth.tiny()
    g = p.geom
    d_obs = orc.forward(g, p.m_true).astype(np.float32).astype(np.float64)
    m32 = p.m_start.astype(np.float32)
    d64 = orc.forward(g, m32)
    trace_err = np.linalg.norm(forward_fp32(g, m32) - d64) / np.linalg.norm(d64)
    resid_ratio = np.linalg.norm(d64 - d_obs) / np.linalg.norm(d_obs)
    assert trace_err < 1.5e-6 and resid_ratio < 2e-3
    e_grad, dev_all, dev_early = _fp32_aa(orc, "kernel", 10)
    assert 5e-4 < e_grad < 3e-3
    assert dev_early < 1e-3           # before the AA extrapolation takes over
    assert 5e-3 < dev_all < 1e-1


@pytest.mark.slow
def test_compensated_fp32_forms_lower_the_trace_floor_to_the_stencils(orc):
    """Carrying the increment, then u as an error-free pair, then u and v as
    pairs: each step lowers the trace error, down to the ~8e-8 that the FP32
    stencil itself leaves (one shot of the tiny problem, start model)."""
    from fp32_emulation import forward_fp32
    p = synth.tiny()
    g = p.geom.subset([0])
    m32 = p.m_start.astype(np.float32)
    d64 = orc.forward(g, m32)
    err = {f: np.linalg.norm(forward_fp32(g, m32, form=f) - d64) / np.linalg.norm(d64)
           for f in ("kernel", "increment", "compensated", "double_uv")}
    assert err["increment"] < 0.3 * err["kernel"]
    assert err["compensated"] < 0.6 * err["increment"]
    assert err["double_uv"] < err["compensated"]
    assert 5e-8 < err["double_uv"] < 1e-7


@pytest.mark.slow
def test_compensated_form_still_misses_the_tiny_targets(orc):
    """The best FP32-field form that keeps single arrays for v (increment form
    with a compensated u) brings the gradient to ~2e-4 but the 10-iteration
    history still departs by more than 1e-2: the tiny problem's targets are
    beyond FP32 wavefields, not an artefact of the kernels' arithmetic."""
    e_grad, dev_all, _ = _fp32_aa(orc, "compensated", 10)
    assert 1e-4 < e_grad < 4e-4
    assert dev_all > 1e-2


@pytest.mark.slow
def test_random_data_noise_barely_moves_the_oracle_history(orc):
    """Random relative perturbations of 1e-7 in the observed data (the size of
    an FP32 trace error) move the oracle's own 10-iteration history by ~2e-5:
    the FP32 departure comes from errors correlated with the model."""
    from oracle import aa
    with open(os.path.join(HERE, "golden", "tiny_aa_history.json")) as f:
        ref = json.load(f)
    p = synth.tiny()
    g = p.geom
    d0 = orc.forward(g, p.m_true)
    d = d0 * (1.0 + 1e-7 * np.random.default_rng(1).standard_normal(d0.shape))
    out = aa.aa_gd(lambda m: orc.fwi_gradient(g, m, d), p.m_start, M=5, eta=ref["eta"], iters=10,
                   bounds=p.m_bounds, misfit_fn=lambda m: 0.5 * float(np.sum((orc.forward(g, m) - d) ** 2)))
    J, Jr = np.array(out["J"]), np.array(ref["J"])
    assert np.linalg.norm(J - Jr) / np.linalg.norm(Jr) < 1e-4


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
