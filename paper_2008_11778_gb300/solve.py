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

import numpy as np
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
                 grad_fn=None, misfit_fn=None, beta=1.0, weights=None, norm=aafwi.NORM_L2):
        """grad_fn(x, g_out, reuse) -> J and misfit_fn(x) -> J replace the wave-
        equation objective (plan / d_obs unused then): Alg. 2 applies to any
        fixed-point map G(p) = p - eta grad J(p).  norm: the norm of the
        optimisation step (Sec. 2.1; aafwi.NORM_L2, NORM_L1 or NORM_LINF)."""
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
            # a zero gradient makes p_0 stationary: any step is the same, keep the factor's scale
            gmax = aafwi.absmax(self.grad)
            eta = eta_factor * aafwi.absmax(self.p) / (gmax if gmax > 0.0 else 1.0)
        self.eta = eta
        self.aa = aafwi.AA(self.p.numel(), M, eta)
        if beta != 1.0:
            self.aa.set_beta(beta)
        if weights is not None:
            self.aa.set_weights(weights.contiguous())
        if norm != aafwi.NORM_L2:
            self.aa.set_norm(norm)
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
           grad_fn=None, misfit_fn=None, beta=1.0, weights=None, norm=aafwi.NORM_L2):
    """Run Alg. 2 for ``iters`` iterations (or until J/J_0 <= target).

    Returns a dict with J (J[k] = J(p_k)), lam, Mk, eta, the final p and grad
    (device), n_forward / n_adjoint pass counts and wall seconds per iteration.
    """
    t0 = time.perf_counter()
    run = AAInversion(plan, d_obs, p0, M, eta, eta_factor, bounds, lambdas, c1, mode, m0, line_search,
                      grad_fn, misfit_fn, beta, weights, norm)
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


# ---------------------------------------------------------------------------
# Comparison solvers of Sec. 5 on the same kernels: L-BFGS(M) and restarted
# GMRES(M).  Vector work runs in the library (aafwi.dot: FP64-accumulated
# inner products; aafwi.axpby); only scalars and the small GMRES
# least-squares problem live on the host.
# ---------------------------------------------------------------------------

class LBFGSInversion(AAInversion):
    """L-BFGS(M) (Sec. 5.2, eqs. secant, lbfgs_update) on the library kernels:

      * direction d = -B_k grad_k by the two-loop recursion over the last M
        pairs (s_i, y_i) = (p_{i+1} - p_i, grad_{i+1} - grad_i), B_0 = gamma I,
        gamma = <s, y>/<y, y> of the newest pair; a pair enters the memory
        only if <s, y> > 0; without a pair d = -eta grad;
      * curvature=False: trial points clip(p + lambda d), lambda in
        (1, 1/2, 1/4, 1/8), the Armijo rule of Alg. 2 (one misfit per trial),
        else the plain gradient step;
      * curvature=True (the Armijo rule plus the curvature condition the paper
        applies in Sec. 4.1): weak Wolfe with c2 = 0.9 by bracketing from
        lambda = 1 (Armijo failing halves, a too-flat slope doubles or
        bisects), one gradient per trial, at most 12 trials, else the last
        Armijo point or the plain gradient step.

    Same state, counters and history as AAInversion (lam = accepted step)."""

    def __init__(self, plan, d_obs, p0, M, curvature=True, c2=0.9, max_trials=12, **kw):
        super().__init__(plan, d_obs, p0, M, **kw)
        self.aa.close()
        self.curvature, self.c2, self.max_trials = curvature, c2, max_trials
        self.S, self.Y, self.rho = [], [], []
        self.d = torch.empty_like(self.p)
        self.g_prev = torch.empty_like(self.p)
        self.g_trial = torch.empty_like(self.p)
        self.p_best = torch.empty_like(self.p)
        self.g_best = torch.empty_like(self.p)
        self.pool = [(torch.empty_like(self.p), torch.empty_like(self.p)) for _ in range(M + 1)]

    def _grad_at(self, x, g_out):
        if self.grad_fn is not None:
            return self.grad_fn(x, g_out, False)
        if self.lsrtm:
            return self.plan.adjoint_gradient(self.mode, self.m0, x, self.d_obs, g_out)
        return self.plan.adjoint_gradient(self.mode, x, None, self.d_obs, g_out)

    def _direction(self):
        """self.d = -B g (two-loop recursion, all vector work in the library)."""
        q = self.d
        q.copy_(self.grad)
        if not self.S:
            aafwi.axpby(0.0, q, -self.eta, q)
            return q
        alphas = []
        for s, y, rho in zip(reversed(self.S), reversed(self.Y), reversed(self.rho)):
            a = rho * aafwi.dot(s, q)
            aafwi.axpby(-a, y, 1.0, q)
            alphas.append(a)
        s, y = self.S[-1], self.Y[-1]
        gamma = aafwi.dot(s, y) / aafwi.dot(y, y)
        aafwi.axpby(0.0, q, gamma, q)
        for (s, y, rho), a in zip(zip(self.S, self.Y, self.rho), reversed(alphas)):
            b = rho * aafwi.dot(y, q)
            aafwi.axpby(a - b, s, 1.0, q)
        aafwi.axpby(0.0, q, -1.0, q)
        return q

    def _trial(self, lam, out):
        """out = clip(p + lam d) (lam = 0: the plain gradient step)."""
        out.copy_(self.p)
        if lam > 0:
            aafwi.axpby_clip(lam, self.d, 1.0, out, self.lo, self.hi)
        else:
            aafwi.axpby_clip(-self.eta, self.grad, 1.0, out, self.lo, self.hi)

    def _armijo(self, Jc, cand):
        diff = self.p_tilde                  # scratch
        diff.copy_(cand)
        aafwi.axpby(-1.0, self.p, 1.0, diff)
        return Jc <= self.J + self.c1 * min(0.0, aafwi.dot(self.grad, diff))

    def _wolfe(self):
        """Weak-Wolfe bracketing along self.d; returns (lam, J) with the point in
        p_best and its gradient in g_best, or None if no trial passed Armijo."""
        lam, lo, hi = 1.0, 0.0, float("inf")
        gd = aafwi.dot(self.grad, self.d)
        best = None
        for _ in range(self.max_trials):
            self._trial(lam, self.cand)
            Jc = self._grad_at(self.cand, self.g_trial)
            self.n_forward += 1
            self.n_adjoint += 1
            if not self._armijo(Jc, self.cand):
                hi = lam
            else:
                best = (lam, Jc)
                self.p_best.copy_(self.cand)
                self.g_best.copy_(self.g_trial)
                if aafwi.dot(self.g_trial, self.d) >= self.c2 * gd:
                    return best
                lo = lam
            lam = 2.0 * lam if hi == float("inf") else 0.5 * (lo + hi)
        return best

    def step(self):
        self._direction()
        self.g_prev.copy_(self.grad)
        lam = 0.0
        if self.curvature:
            hit = self._wolfe()
            if hit is not None:
                lam, J = hit
                self.cand.copy_(self.p_best)
                self.grad.copy_(self.g_best)
            else:
                self._trial(0.0, self.cand)
                J = self._grad_at(self.cand, self.grad)
                self.n_forward += 1
                self.n_adjoint += 1
            self.p, self.cand = self.cand, self.p          # cand now holds p_k
            self.J = J
        else:
            reuse = False
            if self.S:
                for trial in self.lambdas:
                    self._trial(trial, self.cand)
                    Jc = self._misfit_only(self.cand)
                    self.n_forward += 1
                    if self._armijo(Jc, self.cand):
                        lam, reuse = trial, (not self.lsrtm and self.grad_fn is None and self.plan.keeps_forward)
                        break
            if lam == 0.0:
                self._trial(0.0, self.cand)
            self.p, self.cand = self.cand, self.p
            self.J = self._gradient(self.p, reuse)
            if not reuse:
                self.n_forward += 1
            self.n_adjoint += 1
        s, y = self._free_pair()
        s.copy_(self.p)
        aafwi.axpby(-1.0, self.cand, 1.0, s)           # s = p_{k+1} - p_k
        y.copy_(self.grad)
        aafwi.axpby(-1.0, self.g_prev, 1.0, y)         # y = grad_{k+1} - grad_k
        sy = aafwi.dot(s, y)
        if sy > 0.0:
            self.S.append(s)
            self.Y.append(y)
            self.rho.append(1.0 / sy)
            if len(self.S) > self.M:
                self.S.pop(0)
                self.Y.pop(0)
                self.rho.pop(0)
        self.history["J"].append(self.J)
        self.history["lam"].append(lam)
        self.history["Mk"].append(len(self.S))
        self.k += 1
        return self.J

    def _free_pair(self):
        """A buffer pair not held by the memory (the pool has M + 1 pairs, the
        memory at most M)."""
        held = {id(t) for t in self.S}
        for s, y in self.pool:
            if id(s) not in held:
                return s, y
        raise RuntimeError("no free L-BFGS buffer")

    def close(self):
        pass


def lbfgs_fwi(plan, d_obs, p0, M, iters, target=None, **kw):
    """Run LBFGSInversion like aa_fwi (same return layout)."""
    t0 = time.perf_counter()
    run = LBFGSInversion(plan, d_obs, p0, M, **kw)
    ts = [time.perf_counter() - t0]
    for k in range(iters):
        J = run.step()
        ts.append(time.perf_counter() - t0)
        if target is not None and J <= target * run.J0:
            break
    torch.cuda.synchronize()
    out = dict(run.history)
    out.update(eta=run.eta, p=run.p, grad=run.grad, n_forward=run.n_forward, n_adjoint=run.n_adjoint, t=ts)
    return out


def gmres_restarted(residual_fn, x0, M, iters, misfit_fn=None):
    """Restarted GMRES(M) (Sec. 5.1) on the square system A x = b given by its
    residual map residual_fn(x, out) -> out = A x - b (for LSRTM: the LSRTM
    gradient L^T (L x - d), eq. LSRTM3).  One residual evaluation per Arnoldi
    step plus one per restart and one for b; the Krylov basis lives on the
    device, the (M+1) x M Hessenberg least-squares problem on the host (FP64).

    Returns dict(x = last iterate, res = ||b - A x_k|| per step (from the
    small problem), J = misfit_fn(x_k) per step if given, applications)."""
    dev = x0.device
    n = x0.numel()
    V = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(M + 1)]
    w = torch.empty(n, dtype=torch.float32, device=dev)
    zero = torch.zeros_like(x0)
    b = torch.empty(n, dtype=torch.float32, device=dev)
    residual_fn(zero, b)                         # A 0 - b
    aafwi.axpby(0.0, b, -1.0, b)                 # b
    x = x0.detach().to(torch.float32).contiguous().clone().view(-1)
    out = {"res": [], "J": [], "applications": 1}
    done = 0
    while done < iters:
        residual_fn(x.view_as(x0), V[0].view_as(x0))    # A x - b
        out["applications"] += 1
        aafwi.axpby(0.0, V[0], -1.0, V[0])                # r0 = b - A x
        beta = np.sqrt(max(aafwi.dot(V[0], V[0]), 0.0))
        if beta == 0.0:
            break
        aafwi.axpby(0.0, V[0], 1.0 / beta, V[0])
        H = np.zeros((M + 1, M))
        xc = x
        for j in range(M):
            if done == iters:
                break
            residual_fn(V[j].view_as(x0), w.view_as(x0))   # A v - b
            out["applications"] += 1
            aafwi.axpby(1.0, b, 1.0, w)                   # A v
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = aafwi.dot(V[i], w)
                aafwi.axpby(-H[i, j], V[i], 1.0, w)
            H[j + 1, j] = np.sqrt(max(aafwi.dot(w, w), 0.0))
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
            xc = x.clone()
            for i in range(j + 1):
                aafwi.axpby(float(y[i]), V[i], 1.0, xc)
            out["res"].append(float(np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)))
            if misfit_fn is not None:
                out["J"].append(misfit_fn(xc.view_as(x0)))
            done += 1
            if H[j + 1, j] == 0.0:
                break
            aafwi.axpby(0.0, w, 1.0 / H[j + 1, j], w)
            V[j + 1].copy_(w)
        x = xc
    out["x"] = x.view_as(x0)
    return out
