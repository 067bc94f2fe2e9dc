"""The paper's solver comparisons (Sec. 4) on this library's kernels:

  * LSRTM (737 x 240, 64 shots, 4000 steps; start = the RTM image): steepest
    descent, AA(3), L-BFGS(3) and restarted GMRES(3) on the normal equations
    L^T L rho = L^T d (eq. LSRTM3), 20 iterations each;
  * FWI (400 x 150, 32 shots, 2500 steps): steepest descent, AA(10) with the
    l2, l1 and l-infinity norms in its optimisation step (Sec. 2.1) and
    L-BFGS(10), with clean data and with mean-zero uniform noise at an SNR of
    0.55 dB, a fixed budget of gradient evaluations each.

Every run reports J/J0 per iteration, gradient evaluations (adjoint passes),
forward passes and wall seconds on the same GPU.

  python -m paper_2008_11778_gb300.compare [--lsrtm-iters 20] [--fwi-grads 40]
"""
import argparse
import json
import sys
import time

import numpy as np
import torch

from . import aafwi, solve, synth


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _log(*a):
    print(*a, file=sys.stderr, flush=True)


def _timed(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def lsrtm(iters=20, M=3, log=None):
    log = log or _log
    p = synth.lsrtm()
    g = p.geom
    plan = aafwi.Plan(g, 4700.0, l2_batches=1)   # LSRTM reuses no stored forward: L2-sized batches
    m0 = _dev(p.m_true)
    rho_true = _dev(p.extra["rho_true"])
    d = torch.empty(plan.trace_count, device="cuda")
    plan.born_forward(m0, rho_true, d)
    rtm = torch.empty_like(m0)
    plan.born_adjoint(m0, d, rtm)
    dsyn = torch.empty_like(d)

    def J_of(x):
        plan.born_forward(m0, x, dsyn)
        return plan.misfit(dsyn, d)

    J0 = J_of(rtm)
    rows = {}
    for name, Mi in (("steepest_descent", 0), ("aa", M)):
        out, s = _timed(lambda: solve.aa_fwi(plan, d, rtm, M=Mi, iters=iters, mode=aafwi.MODE_LSRTM, m0=m0))
        rows[name] = {"J_over_J0": [j / J0 for j in out["J"]], "gradients": out["n_adjoint"],
                      "forward_passes": out["n_forward"], "seconds": s}
        log(name, rows[name]["J_over_J0"][-1], s)
    for name, curv in (("lbfgs_wolfe", True), ("lbfgs_armijo", False)):
        out, s = _timed(lambda: solve.lbfgs_fwi(plan, d, rtm, M=M, iters=iters, mode=aafwi.MODE_LSRTM, m0=m0,
                                                curvature=curv))
        rows[name] = {"J_over_J0": [j / J0 for j in out["J"]], "gradients": out["n_adjoint"],
                      "forward_passes": out["n_forward"], "seconds": s}
        log(name, rows[name]["J_over_J0"][-1], s)

    def residual_fn(x, o):
        plan.adjoint_gradient(aafwi.MODE_LSRTM, m0, x, d, o, sync=False)

    t0 = time.perf_counter()
    gm = solve.gmres_restarted(residual_fn, rtm, M=M, iters=iters)
    torch.cuda.synchronize()
    s = time.perf_counter() - t0
    Jg = J_of(gm["x"])
    rows["gmres"] = {"normal_residual": [r / gm["res"][0] for r in gm["res"]], "J_over_J0_final": Jg / J0,
                     "operator_applications": gm["applications"], "seconds": s}
    log("gmres", Jg / J0, s)
    return {"workload": "lsrtm-737x240-64shots-4000steps", "iterations": iters, "M": M, "J0": J0, "runs": rows}


def fwi(grads=40, M=10, snr_db=None, log=None):
    log = log or _log
    p = synth.batched()
    g = p.geom
    plan = aafwi.Plan(g, p.c_bounds[1])
    lo, hi = p.m_bounds
    mt = _dev(p.m_true)
    d = torch.empty(plan.trace_count, device="cuda")
    plan.model_forward(mt, d)
    if snr_db is not None:
        d += _dev(synth.uniform_noise(d.cpu().numpy(), snr_db, seed=4 * 1000 + 2008))
    m0 = _dev(p.m_start)
    rows = {}
    norms = {"aa": aafwi.NORM_L2, "aa_l1": aafwi.NORM_L1, "aa_linf": aafwi.NORM_LINF}
    for name in ("steepest_descent", "aa", "aa_l1", "aa_linf", "lbfgs_wolfe", "lbfgs_armijo"):
        if name.startswith("lbfgs"):
            run = solve.LBFGSInversion(plan, d, m0, M, bounds=(lo, hi), curvature=name == "lbfgs_wolfe")
        else:
            run = solve.AAInversion(plan, d, m0, 0 if name == "steepest_descent" else M, bounds=(lo, hi),
                                    norm=norms.get(name, aafwi.NORM_L2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while run.n_adjoint < grads:
            run.step()
        torch.cuda.synchronize()
        s = time.perf_counter() - t0
        rows[name] = {"J_over_J0": [j / run.J0 for j in run.history["J"]], "gradients": run.n_adjoint,
                      "forward_passes": run.n_forward, "seconds": s}
        log(name, rows[name]["J_over_J0"][-1], s)
        run.close()
    return {"workload": "fwi-batched-400x150-32shots-2500steps", "M": M, "snr_db": snr_db,
            "gradient_budget": grads, "runs": rows}


def large_aa(iters=3, M=10, log=None):
    """AA(M) on the large workload (2001 x 601, 200 shots, 6000 steps; the
    planner's shot batches): J/J0 and wall seconds per iteration."""
    log = log or _log
    p = synth.large()
    g = p.geom
    plan = aafwi.Plan(g, p.c_bounds[1])
    lo, hi = p.m_bounds
    d = torch.empty(plan.trace_count, device="cuda")
    plan.model_forward(_dev(p.m_true), d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run = solve.AAInversion(plan, d, _dev(p.m_start), M, bounds=(lo, hi))
    ts = [time.perf_counter() - t0]
    for _ in range(iters):
        run.step()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    out = {"workload": "large-2001x601-200shots-6000steps", "M": M, "shots_per_batch": plan.info.shots_per_batch,
           "batches": plan.info.n_batches, "checkpoint_every": plan.info.checkpoint_every,
           "J_over_J0": [j / run.J0 for j in run.history["J"]], "gradients": run.n_adjoint,
           "forward_passes": run.n_forward, "seconds": ts}
    log("large", out["J_over_J0"][-1], ts[-1])
    run.close()
    return out


def lsrtm_gradient_rate(reps=3, log=None, shots_per_batch=0):
    """Wall time of one LSRTM gradient on the LSRTM workload (737 x 240,
    64 shots, 4000 steps): Born pair forward + adjoint with the background
    replayed from the stored history, timed with CUDA events on the launching
    stream; the rate counts the four wavefield passes per gradient."""
    log = log or _log
    p = synth.lsrtm()
    g = p.geom
    plan = aafwi.Plan(g, 4700.0, shots_per_batch=shots_per_batch, l2_batches=1)
    m0 = _dev(p.m_true)
    rho = _dev(p.extra["rho_true"])
    d = torch.empty(plan.trace_count, device="cuda")
    plan.born_forward(m0, rho, d)
    rho0 = torch.zeros_like(rho)
    grad = torch.empty_like(rho)
    plan.adjoint_gradient(aafwi.MODE_LSRTM, m0, rho0, d, grad)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.adjoint_gradient(aafwi.MODE_LSRTM, m0, rho0, d, grad, sync=False)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    upd = 4 * g.updates_per_pass()
    out = {"workload": "lsrtm-737x240-64shots-4000steps", "ms_per_gradient": min(ms),
           "updates_per_s": upd / (min(ms) * 1e-3), "lanes": plan.info.lanes,
           "checkpoint_every": plan.info.checkpoint_every, "shots_per_batch": plan.info.shots_per_batch}
    log("lsrtm gradient", out["ms_per_gradient"], "ms")
    plan.close()
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser(description="solver comparisons of the paper on this library")
    ap.add_argument("--lsrtm-iters", type=int, default=20)
    ap.add_argument("--fwi-grads", type=int, default=40)
    ap.add_argument("--snr-db", type=float, default=0.55)
    ap.add_argument("--large-iters", type=int, default=0, help="AA iterations on the large workload (0: skip)")
    ap.add_argument("--only-large", action="store_true")
    ap.add_argument("--lsrtm-rate", action="store_true", help="time one LSRTM gradient and stop")
    ap.add_argument("--lsrtm-batch", type=int, default=0,
                    help="shots per batch of the LSRTM plan (0: the planner's L2-sized batches)")
    a = ap.parse_args()
    res = {}
    if a.lsrtm_rate:
        print(json.dumps({"lsrtm_gradient": lsrtm_gradient_rate(shots_per_batch=a.lsrtm_batch)}))
        raise SystemExit(0)
    if not a.only_large:
        res = {"lsrtm": lsrtm(a.lsrtm_iters), "fwi": fwi(a.fwi_grads), "fwi_noisy": fwi(a.fwi_grads, snr_db=a.snr_db)}
    if a.large_iters > 0:
        res["large"] = large_aa(a.large_iters)
    print(json.dumps(res))
