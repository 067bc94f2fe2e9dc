"""FP64 reference of Anderson acceleration for gradient descent (Sec. 2.1, Sec. 3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Contents, each following the paper's statement in its own order:
  aa_alpha         Alg. 1 step 2, eq. AAopt with the l2 norm: constrained
                   weights alpha (sum alpha = 1) from the KKT system.
  aa_update_alpha  Alg. 1 step 3, eq. AAupdate0 with damping beta.
  aa_gamma         eqs. Ak, AAopt2, solveGamma: unconstrained gamma by a
                   Householder QR of the explicit n x M_k matrix (the oracle
                   refactors every iteration; a rank-updated QR as in
                   Sec. 2.1 gives the same factors up to rounding).
  aa_gamma_lp      eq. AAopt with the l1 or l-infinity norm (Sec. 2.1: linear
                   programming), the LP written out on the explicit matrix.
  aa_gd            Alg. 2: l2-AA on the steepest-descent map G(p) = p - eta*grad J(p)
                   (eq. GD) with the backtracking line search between the AA
                   point p~ and the plain point p-bar.
  gmres_full       full-memory GMRES (Sec. 5.1, eqs. Krylov, GMRES), used to
                   pin AA on a linear problem.
  gmres_restarted  restarted GMRES(M) (Sec. 5.1): the Krylov space is rebuilt
                   from the latest iterate every M steps; operator as a function
                   (the LSRTM normal operator L^T L of eq. LSRTM3).
  lbfgs_direction  the L-BFGS two-loop recursion (Sec. 5.2, eqs. secant,
                   lbfgs_update): -B_k g from the last M pairs (s_i, y_i).
  lbfgs            L-BFGS(M) with the backtracking line search of aa_gd.

Readings of points the paper leaves open (shared with the GPU drivers):
  * A_k / f_k are built from the gradients at the last M_k+1 ACCEPTED iterates;
    with a fixed eta the factor -eta cancels, so gamma = argmin||dG g - G_k||.
  * Rank safeguard: while min_j|R_jj| < RANK_TOL * max_j|R_jj| drop the oldest
    column and refactor (the paper is silent).
  * Line search (Alg. 2 step 4): lambda in (1, 1/2, 1/4, 1/8); accept the first
    with J(p_lam) <= J(p_k) + c1*min(0, <grad_k, p_lam - p_k>), c1 = 1e-4;
    otherwise lambda = 0 (the plain gradient step, taken without a test).
  * Bound constraint: after each update p is clipped elementwise to
    [lo, hi] (physical velocity bounds mapped to m = 1/c^2), identically in
    every trial; the Armijo test is applied to the clipped point.
  * Alg. 2 input step p_1 = G(p_0) is taken without a line search.
  * l1 / l-infinity AA: the columns are those the l2 rank safeguard keeps, and
    the weights multiply |residual| (the l2 weights multiply its square).
  * L-BFGS (the paper gives eqs. secant / lbfgs_update, not an algorithm):
    the textbook two-loop recursion with initial matrix gamma_k I,
    gamma_k = <s, y> / <y, y> of the newest pair; a pair enters the memory
    only if <s, y> > 0.  Without a pair the direction is -eta grad.  Line
    search: the paper applies the Armijo rule and the curvature condition
    (Sec. 4.1).  With curvature=False: lambda in (1, 1/2, 1/4, 1/8), the
    same Armijo rule as aa_gd (a misfit per trial), the plain gradient step
    if none passes.  With curvature=True (weak Wolfe, c2 = 0.9; a gradient
    per trial): start at lambda = 1; Armijo failing halves the bracket,
    J(p + lambda d) passing but <grad(p + lambda d), d> < c2 <grad, d>
    doubles lambda (or bisects once bracketed); at most 12 trials, after
    which the last point that passed Armijo is taken (else the plain
    gradient step).  An accepted Wolfe point gives <s, y> > 0.
  * Restarted GMRES(M): the iterate after Arnoldi step j of a cycle is
    x_0 + V_j y_j with y_j minimising ||beta e_1 - H_j y|| (Sec. 5.1); a cycle
    ends after M steps (or on a zero subdiagonal) and the next starts from
    its last iterate.
"""
import numpy as np

RANK_TOL = 1e-6
LAMBDAS = (1.0, 0.5, 0.25, 0.125)
ARMIJO_C1 = 1e-4


# --------------------------------------------------------------------------
# Alg. 1 (general form, used as a pin of the gamma form)
# --------------------------------------------------------------------------

def aa_alpha(F):
    """alpha = argmin ||F alpha||_2 s.t. sum(alpha) = 1   (eq. AAopt, l2 norm).

    KKT system [[2 F^T F, 1], [1^T, 0]] [alpha; mu] = [0; 1].
    """
    F = np.asarray(F, dtype=np.float64)
    m = F.shape[1]
    K = np.zeros((m + 1, m + 1))
    K[:m, :m] = 2.0 * F.T @ F
    K[:m, m] = 1.0
    K[m, :m] = 1.0
    rhs = np.zeros(m + 1)
    rhs[m] = 1.0
    return np.linalg.solve(K, rhs)[:m]


def aa_update_alpha(P, GP, alpha, beta=1.0):
    """eq. AAupdate0: (1-beta) sum alpha_i p_i + beta sum alpha_i G(p_i)."""
    P, GP = np.asarray(P), np.asarray(GP)
    return (1.0 - beta) * (P @ alpha) + beta * (GP @ alpha)


def gamma_to_alpha(gamma):
    """Inverse of gamma_i = alpha_0 + ... + alpha_i (Sec. 2.1), with sum alpha = 1."""
    g = np.concatenate([[0.0], np.asarray(gamma, dtype=np.float64), [1.0]])
    return np.diff(g)


# --------------------------------------------------------------------------
# gamma form (eqs. Ak, AAopt2, solveGamma, AA2_update)
# --------------------------------------------------------------------------

def aa_gamma(A, f, rank_tol=RANK_TOL):
    """Least-squares gamma = argmin ||A gamma - f||_2 by Householder QR.

    Columns of A are ordered oldest first.  Returns (gamma, first) where
    ``first`` is the number of oldest columns dropped by the rank safeguard;
    gamma has A.shape[1] - first entries and refers to A[:, first:].
    """
    A = np.asarray(A, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    first = 0
    while A.shape[1] - first > 0:
        Q, R = np.linalg.qr(A[:, first:], mode="reduced")
        d = np.abs(np.diag(R))
        if d.min() >= rank_tol * d.max() and d.max() > 0.0:
            gamma = np.linalg.solve(R, Q.T @ f) if R.shape[0] > 1 else (Q.T @ f) / R[0, 0]
            return np.atleast_1d(gamma), first
        first += 1
    return np.zeros(0), first


def aa_gamma_lp(A, f, norm, weights=None):
    """gamma = argmin ||W (A gamma - f)||_p for p = 1 ("l1") or infinity
    ("linf"), W = diag(weights) (identity if None): Sec. 2.1 notes that these
    norms in eq. AAopt need linear programming.  The LP is written out on the
    explicit matrix and solved by scipy's HiGHS (the definition, no
    reformulation):
      linf:  min t        s.t.  -t <= w_i (A_i gamma - f_i) <= t
      l1:    min sum e_i  s.t.  -e_i <= w_i (A_i gamma - f_i) <= e_i
    Returns (gamma, optimal value)."""
    from scipy.optimize import linprog
    from scipy.sparse import csr_matrix, hstack, identity, vstack
    A = np.asarray(A, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    n, M = A.shape
    w = np.ones(n) if weights is None else np.asarray(weights, dtype=np.float64)
    Aw, fw = A * w[:, None], f * w
    if norm == "linf":
        one = np.ones((n, 1))
        A_ub = np.block([[Aw, -one], [-Aw, -one]])
        c = np.r_[np.zeros(M), 1.0]
        bounds = [(None, None)] * M + [(0.0, None)]
    elif norm == "l1":
        I = identity(n, format="csr")
        A_ub = vstack([hstack([csr_matrix(Aw), -I]), hstack([csr_matrix(-Aw), -I])]).tocsr()
        c = np.r_[np.zeros(M), np.ones(n)]
        bounds = [(None, None)] * M + [(0.0, None)] * n
    else:
        raise ValueError(norm)
    res = linprog(c, A_ub=A_ub, b_ub=np.r_[fw, -fw], bounds=bounds, method="highs",
                  options={"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10})
    assert res.status == 0, res.message
    gamma = res.x[:M]
    r = np.abs(w * (A @ gamma - f))
    return gamma, float(r.max() if norm == "linf" else r.sum())


def anderson_point(P, Gr, eta, rank_tol=RANK_TOL, beta=1.0, weights=None, norm="l2"):
    """Alg. 2 steps 1-3 for the history P = [p_{k-Mk}..p_k], Gr = [G_{k-Mk}..G_k].

    With a damping beta != 1 the AA point is Alg. 1's eq. AAupdate0,
    (1 - beta) sum_i alpha_i p_i + beta sum_i alpha_i G(p_i), with alpha from
    gamma (the same weights); beta = 1 is Alg. 2's step 3 below.
    weights: the diagonal of a weighted l2 norm for the least squares of step 2
    (Sec. 2.1 admits other norms): gamma = argmin sum_i w_i (dG gamma - G_k)_i^2.

    Returns (p_bar, p_tilde, gamma, Mk_used).
      p_bar   = G(p_k) = p_k - eta G_k                         (step 1, eq. GD)
      gamma   = argmin || [G_{i+1} - G_i] gamma - G_k ||        (step 2; the -eta of
                 f_k = -eta G_k and A_k = -eta [dG] cancels; the l2 norm
                 unless norm is "l1" or "linf", see aa_gamma_lp)
      p_tilde = G(p_k) - sum_i gamma_i [G(p_{i+1}) - G(p_i)]   (step 3, eq. AA2_update)
    """
    shape = np.shape(P[-1])
    P = [np.asarray(p, dtype=np.float64).ravel() for p in P]
    Gr = [np.asarray(g, dtype=np.float64).ravel() for g in Gr]
    gk = Gr[-1]
    p_bar = P[-1] - eta * gk
    Mk = len(P) - 1
    if Mk == 0:
        return p_bar.reshape(shape), p_bar.reshape(shape).copy(), np.zeros(0), 0
    dG = np.stack([Gr[i + 1] - Gr[i] for i in range(Mk)], axis=1)
    if weights is None:
        gamma, first = aa_gamma(dG, gk, rank_tol)
    else:
        sw = np.sqrt(np.asarray(weights, dtype=np.float64).ravel())
        gamma, first = aa_gamma(dG * sw[:, None], gk * sw, rank_tol)
    if norm != "l2" and len(gamma):
        # l1 / l-infinity (Sec. 2.1) over the columns the l2 rank safeguard keeps
        gamma, _ = aa_gamma_lp(dG[:, first:], gk, norm, weights)
    if beta != 1.0:
        Pk, Gk = P[first:], Gr[first:]
        alpha = gamma_to_alpha(gamma)
        p_tilde = aa_update_alpha(np.stack(Pk, axis=1), np.stack([p - eta * g for p, g in zip(Pk, Gk)], axis=1),
                                  alpha, beta)
        return p_bar.reshape(shape), np.asarray(p_tilde).reshape(shape), gamma, Mk - first
    p_tilde = p_bar.copy()
    for j, gj in enumerate(gamma):
        i = first + j
        dGp = (P[i + 1] - eta * Gr[i + 1]) - (P[i] - eta * Gr[i])
        p_tilde -= gj * dGp
    return p_bar.reshape(shape), p_tilde.reshape(shape), gamma, Mk - first


def aa_gd(grad_fn, p0, M, eta, iters, line_search=True, bounds=None,
          lambdas=LAMBDAS, c1=ARMIJO_C1, rank_tol=RANK_TOL, misfit_fn=None, beta=1.0, weights=None,
          norm="l2"):
    """Alg. 2: l2-based AA for gradient descent.

    grad_fn(p) -> (J, grad); misfit_fn(p) -> J (defaults to grad_fn(p)[0]).
    Iteration k = 0 is the input step p_1 = G(p_0); iterations k >= 1 are
    Alg. 2 steps 1-5.  Returns a dict with the accepted iterates ``p``, their
    misfits ``J`` (J[k] = J(p_k), len iters+1), ``lam`` and ``Mk`` per
    iteration and the number of misfit-only evaluations ``n_trials``.
    """
    if misfit_fn is None:
        misfit_fn = lambda p: grad_fn(p)[0]
    clip = (lambda p: np.clip(p, bounds[0], bounds[1])) if bounds is not None else (lambda p: p)
    p = np.asarray(p0, dtype=np.float64).copy()
    J, g = grad_fn(p)
    P, Gr = [p], [g]
    out = {"p": [p], "J": [J], "lam": [], "Mk": [], "gamma": [], "n_trials": 0}
    for k in range(iters):
        if k == 0:
            p_next = clip(p - eta * g)       # Alg. 2 input: p_1 = G(p_0)
            lam, Mk, gamma = 0.0, 0, np.zeros(0)
        else:
            p_bar, p_tilde, gamma, Mk = anderson_point(P, Gr, eta, rank_tol, beta, weights, norm)
            lam = 0.0
            if line_search and Mk > 0:
                for trial in lambdas:
                    cand = clip(trial * p_tilde + (1.0 - trial) * p_bar)
                    Jc = misfit_fn(cand)
                    out["n_trials"] += 1
                    if Jc <= J + c1 * min(0.0, float(np.vdot(g, cand - p))):
                        lam = trial
                        break
            elif not line_search:
                lam = 1.0
            p_next = clip(lam * p_tilde + (1.0 - lam) * p_bar)
        p = p_next
        J, g = grad_fn(p)
        P.append(p)
        Gr.append(g)
        if len(P) > M + 1:
            P.pop(0)
            Gr.pop(0)
        out["p"].append(p)
        out["J"].append(J)
        out["lam"].append(lam)
        out["Mk"].append(Mk)
        out["gamma"].append(gamma)
    return out


# --------------------------------------------------------------------------
# Full-memory GMRES (Sec. 5.1)
# --------------------------------------------------------------------------

def gmres_full(A, b, x0, kmax):
    """Iterates x_1..x_kmax of GMRES on A x = b: x_k = x0 + V_k y_k minimising
    ||b - A x_k||_2 over the Krylov space K_k(A, r_0) (Arnoldi with modified
    Gram-Schmidt; the small least-squares problem by a library lstsq)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    r0 = b - A @ x0
    beta = np.linalg.norm(r0)
    V = np.zeros((n, kmax + 1))
    H = np.zeros((kmax + 1, kmax))
    V[:, 0] = r0 / beta
    xs = []
    for k in range(kmax):
        w = A @ V[:, k]
        for i in range(k + 1):
            H[i, k] = V[:, i] @ w
            w = w - H[i, k] * V[:, i]
        H[k + 1, k] = np.linalg.norm(w)
        if H[k + 1, k] > 0:
            V[:, k + 1] = w / H[k + 1, k]
        e1 = np.zeros(k + 2)
        e1[0] = beta
        y = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)[0]
        xs.append(x0 + V[:, :k + 1] @ y)
    return xs


# --------------------------------------------------------------------------
# Restarted GMRES(M) (Sec. 5.1)
# --------------------------------------------------------------------------

def gmres_restarted(apply_A, b, x0, M, iters):
    """Restarted GMRES(M) on A x = b with A given as a function.  Returns the
    iterates after each Arnoldi step (iters of them, one operator application
    each) and the residual norms ||b - A x|| the small problem predicts."""
    shape = np.shape(x0)                          # unknowns of any shape, handled as flat vectors
    A = lambda v: np.asarray(apply_A(v.reshape(shape)), dtype=np.float64).ravel()
    x = np.asarray(x0, dtype=np.float64).ravel().copy()
    b = np.asarray(b, dtype=np.float64).ravel()
    xs, res = [], []
    done = 0
    while done < iters:
        r0 = b - A(x)
        beta = np.linalg.norm(r0)
        if beta == 0.0:
            xs += [x.reshape(shape).copy()] * (iters - done)
            res += [0.0] * (iters - done)
            break
        V = [r0 / beta]
        H = np.zeros((M + 1, M))
        xc = x
        for j in range(M):
            if done == iters:
                break
            w = A(V[j])
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = float(np.vdot(V[i], w))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
            xc = x + np.column_stack(V[:j + 1]) @ y
            xs.append(xc.reshape(shape))
            res.append(float(np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)))
            done += 1
            if H[j + 1, j] == 0.0:
                break
            V.append(w / H[j + 1, j])
        x = xc
    return xs, res


# --------------------------------------------------------------------------
# L-BFGS(M) (Sec. 5.2)
# --------------------------------------------------------------------------

def lbfgs_direction(g, S, Y):
    """-B g by the two-loop recursion from the pairs (S[i], Y[i]), oldest
    first; B_0 = gamma I with gamma = <s, y>/<y, y> of the newest pair."""
    q = np.asarray(g, dtype=np.float64).copy()
    a = []
    for s, y in zip(reversed(S), reversed(Y)):
        rho = 1.0 / float(np.vdot(y, s))
        ai = rho * float(np.vdot(s, q))
        q = q - ai * y
        a.append((rho, ai))
    gamma = float(np.vdot(S[-1], Y[-1]) / np.vdot(Y[-1], Y[-1])) if S else 1.0
    r = gamma * q
    for (s, y), (rho, ai) in zip(zip(S, Y), reversed(a)):
        bi = rho * float(np.vdot(y, r))
        r = r + (ai - bi) * s
    return -r


def _wolfe_search(grad_fn, p, J, g, d, clip, c1, c2, max_trials, out):
    """Weak-Wolfe bracketing search along d (see the readings); returns
    (lambda, p_new, J_new, g_new) or None if no trial passed Armijo."""
    lam, lo, hi = 1.0, 0.0, np.inf
    gd = float(np.vdot(g, d))
    best = None
    for _ in range(max_trials):
        cand = clip(p + lam * d)
        Jc, gc = grad_fn(cand)
        out["n_trials"] += 1
        if not Jc <= J + c1 * min(0.0, float(np.vdot(g, cand - p))):
            hi = lam
        else:
            best = (lam, cand, Jc, gc)
            if float(np.vdot(gc, d)) >= c2 * gd:
                return best
            lo = lam
        lam = 2.0 * lam if hi == np.inf else 0.5 * (lo + hi)
    return best


def lbfgs(grad_fn, p0, M, eta, iters, bounds=None, lambdas=LAMBDAS, c1=ARMIJO_C1, misfit_fn=None,
          curvature=False, c2=0.9, max_trials=12):
    """L-BFGS(M) with the readings above; same return layout as aa_gd (lam =
    the accepted step, 0 for a plain gradient step; n_trials counts misfit
    evaluations, or gradient evaluations with curvature=True)."""
    if misfit_fn is None:
        misfit_fn = lambda p: grad_fn(p)[0]
    clip = (lambda p: np.clip(p, bounds[0], bounds[1])) if bounds is not None else (lambda p: p)
    p = np.asarray(p0, dtype=np.float64).copy()
    J, g = grad_fn(p)
    S, Y = [], []
    out = {"p": [p], "J": [J], "lam": [], "n_trials": 0}
    for k in range(iters):
        lam = 0.0
        d = lbfgs_direction(g, S, Y) if S else -eta * g
        if curvature:
            hit = _wolfe_search(grad_fn, p, J, g, d, clip, c1, c2, max_trials, out)
            if hit is not None:
                lam, p_next, J_next, g_next = hit
            else:
                p_next = clip(p - eta * g)
                J_next, g_next = grad_fn(p_next)
        else:
            if S:
                for trial in lambdas:
                    cand = clip(p + trial * d)
                    Jc = misfit_fn(cand)
                    out["n_trials"] += 1
                    if Jc <= J + c1 * min(0.0, float(np.vdot(g, cand - p))):
                        lam = trial
                        break
            p_next = clip(p + lam * d) if lam > 0 else clip(p - eta * g)
            J_next, g_next = grad_fn(p_next)
        s, y = p_next - p, g_next - g
        if float(np.vdot(s, y)) > 0.0:
            S.append(s)
            Y.append(y)
            if len(S) > M:
                S.pop(0)
                Y.pop(0)
        p, J, g = p_next, J_next, g_next
        out["p"].append(p)
        out["J"].append(J)
        out["lam"].append(lam)
    return out
