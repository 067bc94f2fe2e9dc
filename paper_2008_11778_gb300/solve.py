"""Alg. 2 (l2-based Anderson acceleration for gradient descent) driven on the GPU.

Host code decides only control flow (which lambda to try, when to stop); every
vector operation, wave solve and reduction runs in libaafwi.so kernels.

Readings of the points the paper leaves open (the FP64 oracle uses the same):
  * eta = eta_factor * max|p_0| / max|grad J(p_0)|, fixed afterwards (eq. GD).
  * History = last M+1 accepted iterates and their gradients (Sec. 5.1 sliding
    window); gamma from the FP64 Gram matrix with the rank safeguard of the
    library (drop the oldest column while min R_jj < 1e-6 max R_jj).
  * Line search (Alg. 2 step 4): lambda in (1, 1/2, 1/4, 1/8), accept the first
    with J(p_lam) <= J(p_k) + 1e-4 min(0, <grad_k, p_lam - p_k>); otherwise
    lambda = 0 (the plain gradient step, no test).  Every trial point is
    clipped to the bounds before it is evaluated.
  * Iteration 0 is the input step p_1 = G(p_0) (no line search).

The accepted trial's forward wavefield stays in the plan, so the gradient at
the new iterate only runs the adjoint sweep (AAFWI_REUSE_FORWARD).
"""
import time

import torch

from . import aafwi

LAMBDAS = (1.0, 0.5, 0.25, 0.125)
ARMIJO_C1 = 1e-4


class AAInversion:
    """State of one Alg. 2 run; ``step()`` performs one iteration.

    FWI: p = m (device [nz, nx] float32), d_obs the observed traces.
    LSRTM: p = rho with background m0 (mode=MODE_LSRTM).
    Counters: n_forward / n_adjoint wave passes so far (each pass = one sweep
    of every shot over its record).
    """

    def __init__(self, plan, d_obs, p0, M, eta=None, eta_factor=1e-4, bounds=None,
                 lambdas=LAMBDAS, c1=ARMIJO_C1, mode=aafwi.MODE_FWI, m0=None, line_search=True,
                 grad_fn=None, misfit_fn=None):
        """grad_fn(x, g_out, reuse) -> J and misfit_fn(x) -> J replace the wave-
        equation objective (plan / d_obs unused then): Alg. 2 applies to any
        fixed-point map G(p) = p - eta grad J(p)."""
        self.plan, self.d_obs, self.M = plan, d_obs, M
        self.grad_fn, self.misfit_fn = grad_fn, misfit_fn
        self.mode, self.m0 = mode, m0
        self.lsrtm = mode == aafwi.MODE_LSRTM
        self.lo, self.hi = (float(bounds[0]), float(bounds[1])) if bounds is not None else (0.0, 0.0)
        self.lambdas, self.c1, self.line_search = lambdas, c1, line_search
        self.p = p0.detach().to(torch.float32).contiguous().clone()
        self.cand = torch.empty_like(self.p)
        self.grad = torch.empty_like(self.p)
        self.p_tilde = torch.empty_like(self.p)
        self.p_bar = torch.empty_like(self.p)
        self.dsyn = (torch.empty(plan.trace_count, dtype=torch.float32, device=self.p.device)
                     if plan is not None else None)
        self.J = self._gradient(self.p, False)
        self.J0 = self.J
        self.n_forward, self.n_adjoint = 1, 1
        if eta is None:
            eta = eta_factor * aafwi.absmax(self.p) / aafwi.absmax(self.grad)
        self.eta = eta
        self.aa = aafwi.AA(self.p.numel(), M, eta)
        self.k = 0
        self.history = {"J": [self.J], "lam": [], "Mk": []}

    def _gradient(self, x, reuse):
        if self.grad_fn is not None:
            return self.grad_fn(x, self.grad, reuse)
        if self.lsrtm:
            return self.plan.adjoint_gradient(self.mode, self.m0, x, self.d_obs, self.grad)
        return self.plan.adjoint_gradient(self.mode, x, None, self.d_obs, self.grad, reuse_forward=reuse)

    def _misfit_only(self, x):
        if self.misfit_fn is not None:
            return self.misfit_fn(x)
        if self.lsrtm:
            self.plan.born_forward(self.m0, x, self.dsyn)
        else:
            self.plan.model_forward(x, self.dsyn)
        return self.plan.misfit(self.dsyn, self.d_obs)

    def step(self):
        """One iteration of Alg. 2; returns J(p_{k+1})."""
        _, Mk = self.aa.step(self.p, self.grad, self.p_tilde, self.p_bar, want_gamma=True)
        lam, reuse = 0.0, False
        if self.k > 0 and Mk > 0:
            if self.line_search:
                for trial in self.lambdas:
                    dot = self.aa.combine(trial, self.p_tilde, self.p_bar, self.cand, self.lo, self.hi,
                                          want_dot=True)
                    Jc = self._misfit_only(self.cand)
                    self.n_forward += 1
                    if Jc <= self.J + self.c1 * min(0.0, dot):
                        # a plan that runs its shots in batches keeps no forward to reuse
                        lam, reuse = trial, (not self.lsrtm and self.grad_fn is None
                                             and self.plan.keeps_forward)
                        break
            else:
                lam = 1.0
        if lam == 0.0 or not self.line_search:
            self.aa.combine(lam, self.p_tilde, self.p_bar, self.cand, self.lo, self.hi)
            reuse = False
        self.p, self.cand = self.cand, self.p
        self.J = self._gradient(self.p, reuse)
        if not reuse:
            self.n_forward += 1
        self.n_adjoint += 1
        self.history["J"].append(self.J)
        self.history["lam"].append(lam)
        self.history["Mk"].append(Mk if self.k > 0 else 0)
        self.k += 1
        return self.J

    def close(self):
        self.aa.close()


def aa_fwi(plan, d_obs, p0, M, iters, eta=None, eta_factor=1e-4, bounds=None, lambdas=LAMBDAS,
           c1=ARMIJO_C1, mode=aafwi.MODE_FWI, m0=None, line_search=True, target=None, callback=None,
           grad_fn=None, misfit_fn=None):
    """Run Alg. 2 for ``iters`` iterations (or until J/J_0 <= target).

    Returns a dict with J (J[k] = J(p_k)), lam, Mk, eta, the final p and grad
    (device), n_forward / n_adjoint pass counts and wall seconds per iteration.
    """
    t0 = time.perf_counter()
    run = AAInversion(plan, d_obs, p0, M, eta, eta_factor, bounds, lambdas, c1, mode, m0, line_search,
                      grad_fn, misfit_fn)
    ts = [time.perf_counter() - t0]
    for k in range(iters):
        J = run.step()
        ts.append(time.perf_counter() - t0)
        if callback:
            callback(k, run.p, run.grad, J)
        if target is not None and J <= target * run.J0:
            break
    torch.cuda.synchronize()
    out = dict(run.history)
    out.update(eta=run.eta, p=run.p, grad=run.grad, n_forward=run.n_forward, n_adjoint=run.n_adjoint, t=ts)
    run.close()
    return out
