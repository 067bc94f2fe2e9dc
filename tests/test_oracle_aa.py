"""Pins of the FP64 Anderson-acceleration oracle (oracle/aa.py), CPU only.

Checked against: plain steepest descent (M = 0, Sec. 2.1), the Picard bound
(Sec. 2.1), the constrained alpha form (eq. AAopt, solved through its KKT
system), the multi-secant characterisation (Sec. 5.2, eqs. aa_secant_update,
aaFnorm, multisecant), an SVD least-squares solver, and full-memory GMRES on a
linear problem (Sec. 5.1; Walker & Ni 2011: x_AA(k+1) = G(x_GMRES(k))).
"""
import numpy as np
import pytest

from oracle import aa


def _quadratic(n=30, seed=0, cond=50.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, cond, n)) @ Q.T
    b = rng.standard_normal(n)

    def grad_fn(x):
        return 0.5 * x @ A @ x - b @ x, A @ x - b
    return A, b, grad_fn


def test_memory_zero_is_steepest_descent_bitwise():
    A, b, gf = _quadratic()
    eta = 1.0 / 50.0
    x0 = np.zeros(30)
    out = aa.aa_gd(gf, x0, M=0, eta=eta, iters=15)
    x = x0.copy()
    for k in range(15):
        x = x - eta * (A @ x - b)
        assert np.array_equal(out["p"][k + 1], x)


def test_fixed_point_iff_zero_gradient():
    A, b, gf = _quadratic()
    xs = np.linalg.solve(A, b)
    _, g = gf(xs)
    assert np.linalg.norm((xs - 0.01 * g) - xs) < 1e-12


def test_gamma_equals_alpha_form_and_update():
    rng = np.random.default_rng(1)
    n, m = 50, 6
    F = rng.standard_normal((n, m + 1))          # f_{k-m} .. f_k
    P = rng.standard_normal((n, m + 1))
    GP = P + F                                   # G(p_i) = p_i + f_i
    alpha = aa.aa_alpha(F)
    assert alpha.sum() == pytest.approx(1.0, abs=1e-14)
    A = np.diff(F, axis=1)                       # eq. Ak
    gamma, first = aa.aa_gamma(A, F[:, -1])
    assert first == 0
    np.testing.assert_allclose(aa.gamma_to_alpha(gamma), alpha, rtol=1e-10, atol=1e-12)
    upd_alpha = aa.aa_update_alpha(P, GP, alpha, beta=1.0)
    upd_gamma = GP[:, -1] - np.diff(GP, axis=1) @ gamma    # eq. AA2_update
    np.testing.assert_allclose(upd_gamma, upd_alpha, rtol=1e-10, atol=1e-12)
    # AA is never worse than Picard: ||F alpha|| <= ||f_k||
    assert np.linalg.norm(F @ alpha) <= np.linalg.norm(F[:, -1]) + 1e-14


def test_gamma_matches_svd_least_squares():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((200, 8))
    f = rng.standard_normal(200)
    g, first = aa.aa_gamma(A, f)
    ref = np.linalg.lstsq(A, f, rcond=None)[0]
    assert first == 0
    np.testing.assert_allclose(g, ref, rtol=1e-11, atol=1e-13)


def test_rank_safeguard_drops_oldest_column():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 4))
    A[:, 0] = A[:, 2] * 3.0 + 1e-9 * rng.standard_normal(40)   # oldest column nearly dependent
    f = rng.standard_normal(40)
    g, first = aa.aa_gamma(A, f)
    assert first == 1 and len(g) == 3
    np.testing.assert_allclose(g, np.linalg.lstsq(A[:, 1:], f, rcond=None)[0], rtol=1e-10)


def test_picard_bound_along_an_aa_run():
    A, b, gf = _quadratic(seed=4)
    eta = 1.0 / 50.0
    out = aa.aa_gd(gf, np.zeros(30), M=4, eta=eta, iters=12, line_search=False)
    ps = out["p"]
    for k in range(1, 12):
        lo = max(0, k - 4)
        F = np.stack([-eta * gf(p)[1] for p in ps[lo:k + 1]], axis=1)
        gamma = out["gamma"][k]
        alpha = aa.gamma_to_alpha(gamma)
        Fa = F[:, F.shape[1] - len(alpha):] @ alpha
        assert np.linalg.norm(Fa) <= np.linalg.norm(F[:, -1]) * (1 + 1e-12)


def test_multisecant_characterisation():
    """p_tilde = p_k - S_k f_k with S_k = -I + (P+D) D^+ : S_k D_k = P_k and S_k
    has the least ||S + I||_F among all solutions (Sec. 5.2)."""
    A, b, gf = _quadratic(n=25, seed=5)
    eta = 0.02
    rng = np.random.default_rng(5)
    Ps = [rng.standard_normal(25) for _ in range(5)]
    Gs = [gf(p)[1] for p in Ps]
    p_bar, p_tilde, gamma, Mk = aa.anderson_point(Ps, Gs, eta)
    assert Mk == 4
    fs = [-eta * g for g in Gs]
    Pm = np.stack([Ps[i + 1] - Ps[i] for i in range(4)], axis=1)
    Dm = np.stack([fs[i + 1] - fs[i] for i in range(4)], axis=1)
    S = -np.eye(25) + (Pm + Dm) @ np.linalg.pinv(Dm)
    np.testing.assert_allclose(S @ Dm, Pm, atol=1e-10)
    np.testing.assert_allclose(Ps[-1] - S @ fs[-1], p_tilde, rtol=1e-9, atol=1e-11)
    # any other solution S + E with E D = 0 is farther from -I
    E = rng.standard_normal((25, 25))
    E = E - E @ Dm @ np.linalg.pinv(Dm)
    assert np.linalg.norm(S + E + np.eye(25)) > np.linalg.norm(S + np.eye(25))


def test_gmres_oracle_solves_in_n_steps():
    A, b, _ = _quadratic(n=8, seed=6)
    xs = aa.gmres_full(A, b, np.zeros(8), 8)
    res = [np.linalg.norm(A @ x - b) for x in xs]
    assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(7))
    assert res[-1] < 1e-10 * np.linalg.norm(b)


def test_full_memory_aa_is_gmres_mapped_by_G():
    """Sec. 2.1 / 5.1: with M = infinity, beta = 1 and no line search, AA on
    G(x) = x - eta (A x - b) satisfies x_AA(k+1) = G(x_GMRES(k))."""
    n, K = 30, 10
    A, b, gf = _quadratic(n=n, seed=7)
    eta = 1.0 / 50.0
    x0 = np.zeros(n)
    out = aa.aa_gd(gf, x0, M=100, eta=eta, iters=K, line_search=False)
    xg = aa.gmres_full(A, b, x0, K)
    G = lambda x: x - eta * (A @ x - b)
    for k in range(1, K):
        ref = G(xg[k - 1])
        assert np.linalg.norm(out["p"][k + 1] - ref) <= 1e-9 * np.linalg.norm(ref)


def test_line_search_keeps_misfit_monotone_and_beats_sd():
    A, b, gf = _quadratic(seed=8, cond=200.0)
    eta = 1.0 / 200.0
    out = aa.aa_gd(gf, np.zeros(30), M=5, eta=eta, iters=30)
    J = np.array(out["J"])
    assert (np.diff(J[1:]) <= 1e-12 * np.abs(J[1:-1])).all()
    sd = aa.aa_gd(gf, np.zeros(30), M=0, eta=eta, iters=30)
    Jstar = gf(np.linalg.solve(A, b))[0]
    assert (J[-1] - Jstar) < 1e-3 * (sd["J"][-1] - Jstar)


# ---------------------------------------------------- restarted GMRES, L-BFGS

def test_restarted_gmres_without_restart_is_full_gmres():
    rng = np.random.default_rng(21)
    n = 30
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    xs, res = aa.gmres_restarted(lambda v: A @ v, b, x0, M=12, iters=12)
    ref = aa.gmres_full(A, b, x0, 12)
    for a, r in zip(xs, ref):
        np.testing.assert_allclose(a, r, rtol=1e-10, atol=1e-12)
    for x, r in zip(xs, res):
        assert abs(np.linalg.norm(b - A @ x) - r) <= 1e-9 * np.linalg.norm(b)


def test_restarted_gmres_cycles_minimise_over_their_krylov_space():
    """Each iterate minimises ||b - A x|| over x_cycle + K_j(A, r_cycle) --
    checked against a least-squares solve over the explicit (non-Arnoldi)
    Krylov basis -- and the residual never grows across restarts."""
    rng = np.random.default_rng(22)
    n, M = 40, 3
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, 50.0, n)) @ Q.T
    b = rng.standard_normal(n)
    xs, res = aa.gmres_restarted(lambda v: A @ v, b, np.zeros(n), M=M, iters=12)
    assert all(r2 <= r1 * (1 + 1e-12) for r1, r2 in zip(res, res[1:]))
    x_cycle = np.zeros(n)
    for c in range(4):
        r0 = b - A @ x_cycle
        K = np.column_stack([np.linalg.matrix_power(A, i) @ r0 for i in range(M)])
        for j in range(1, M + 1):
            y = np.linalg.lstsq(A @ K[:, :j], r0, rcond=None)[0]
            best = x_cycle + K[:, :j] @ y
            np.testing.assert_allclose(xs[c * M + j - 1], best, rtol=1e-7, atol=1e-9)
        x_cycle = xs[c * M + M - 1]


def test_two_loop_recursion_is_the_dense_bfgs_update():
    """-B g from the two-loop recursion equals the product of explicit BFGS
    inverse updates H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T from
    gamma I, and the newest secant condition B y_k = s_k holds."""
    rng = np.random.default_rng(23)
    n, m = 25, 5
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, 20.0, n)) @ Q.T
    S = [rng.standard_normal(n) for _ in range(m)]
    Y = [A @ s for s in S]                        # curvature pairs of a convex quadratic
    g = rng.standard_normal(n)
    gamma = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1])
    H = gamma * np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / (y @ s)
        E = np.eye(n) - rho * np.outer(s, y)
        H = E @ H @ E.T + rho * np.outer(s, s)
    np.testing.assert_allclose(aa.lbfgs_direction(g, S, Y), -H @ g, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(-aa.lbfgs_direction(Y[-1], S, Y), S[-1], rtol=1e-10, atol=1e-12)


def test_lbfgs_monotone_and_reaches_the_quadratic_minimiser():
    rng = np.random.default_rng(24)
    n = 60
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, 100.0, n)) @ Q.T
    b = rng.standard_normal(n)
    gf = lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b)
    out = aa.lbfgs(gf, np.zeros(n), M=10, eta=1.0 / 100.0, iters=60)
    J = np.array(out["J"])
    assert np.all(np.diff(J) <= 1e-12 * abs(J[0]) + 1e-15)
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(out["p"][-1] - xs) < 1e-6 * np.linalg.norm(xs)
    assert sum(l == 1.0 for l in out["lam"]) >= len(out["lam"]) // 2   # mostly full steps


def test_lbfgs_wolfe_search_keeps_curvature_on_a_nonconvex_start():
    """On f(x) = sum(x^4)/4 - |x|^2/2 started near the local maximum at 0
    (negative curvature along -grad), fixed small gradient steps give no pair
    with <s, y> > 0 and the Armijo-only run never leaves steepest descent;
    the weak-Wolfe search expands the step past the concave region, builds
    pairs and reaches a minimiser (|x_i| = 1)."""
    rng = np.random.default_rng(25)
    n = 20
    x0 = 1e-3 * rng.standard_normal(n)
    f = lambda x: (0.25 * np.sum(x ** 4) - 0.5 * x @ x, x ** 3 - x)
    eta = 1e-3
    x1 = x0 - eta * f(x0)[1]
    assert (x1 - x0) @ (f(x1)[1] - f(x0)[1]) < 0            # a plain step has no usable pair
    out = aa.lbfgs(f, x0, M=5, eta=eta, iters=40, curvature=True)
    J = np.array(out["J"])
    assert np.all(np.diff(J) <= 1e-12)
    assert np.allclose(np.abs(out["p"][-1]), 1.0, atol=1e-4)
    pairs = sum((q - p) @ (f(q)[1] - f(p)[1]) > 0 for p, q in zip(out["p"], out["p"][1:]))
    assert pairs >= len(out["lam"]) // 2
    plain = aa.lbfgs(f, x0, M=5, eta=eta, iters=40, curvature=False)
    assert all(l == 0.0 for l in plain["lam"]) and plain["J"][-1] > 0.5 * J[-1]


def test_damped_anderson_point():
    """beta = 1 of eq. AAupdate0 is Alg. 2's gamma form; beta = 0 is the same
    combination of the iterates alone; any beta is the gamma form with the
    step eta scaled by beta, p_k - beta eta G_k - sum gamma (dp - beta eta dG)."""
    rng = np.random.default_rng(26)
    n, m, eta = 50, 4, 0.1
    P = [rng.standard_normal(n) for _ in range(m + 1)]
    Gr = [rng.standard_normal(n) for _ in range(m + 1)]
    pb, pt1, gam, Mk = aa.anderson_point(P, Gr, eta)
    assert Mk == m                                     # full rank: no column dropped
    GP = np.stack([p - eta * g for p, g in zip(P, Gr)], axis=1)
    pt1b = aa.aa_update_alpha(np.stack(P, axis=1), GP, aa.gamma_to_alpha(gam), 1.0)
    np.testing.assert_allclose(pt1b, pt1, rtol=1e-10, atol=1e-12)
    for beta in (0.0, 0.3, 0.75):
        _, ptb, g, _ = aa.anderson_point(P, Gr, eta, beta=beta)
        ref = P[-1] - beta * eta * Gr[-1]
        for j in range(len(g)):
            ref = ref - g[j] * ((P[j + 1] - beta * eta * Gr[j + 1]) - (P[j] - beta * eta * Gr[j]))
        np.testing.assert_allclose(ptb, ref, rtol=1e-10, atol=1e-12)
    assert np.allclose(pb, P[-1] - eta * Gr[-1])


def test_weighted_l2_gamma():
    """A constant weight leaves gamma unchanged (scale invariance of the
    minimiser); a 0/1 weight gives the gamma of the selected rows alone."""
    rng = np.random.default_rng(27)
    n, m, eta = 80, 4, 0.1
    P = [rng.standard_normal(n) for _ in range(m + 1)]
    Gr = [rng.standard_normal(n) for _ in range(m + 1)]
    _, pt, g0, _ = aa.anderson_point(P, Gr, eta)
    _, ptc, gc, _ = aa.anderson_point(P, Gr, eta, weights=np.full(n, 7.5))
    np.testing.assert_allclose(gc, g0, rtol=1e-10)
    np.testing.assert_allclose(ptc, pt, rtol=1e-10)
    sel = rng.random(n) < 0.5
    _, _, gs, _ = aa.anderson_point(P, Gr, eta, weights=sel.astype(float))
    _, _, gr, _ = aa.anderson_point([p[sel] for p in P], [g[sel] for g in Gr], eta)
    np.testing.assert_allclose(gs, gr, rtol=1e-10)


# ------------------------------------------------- l1 / l-infinity AA (Sec. 2.1)

def _lp_data(n, M, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, M))
    f = A @ rng.standard_normal(M) + rng.laplace(size=n)
    return A, f


def test_l1_gamma_is_the_weighted_median_for_one_column():
    """M = 1: argmin sum |a_i g - f_i| = sum |a_i| |g - f_i/a_i| is the median
    of the ratios f_i/a_i weighted by |a_i| (closed form)."""
    from oracle import aa
    A, f = _lp_data(41, 1, 1)
    a = A[:, 0]
    ratio, wgt = f / a, np.abs(a)
    order = np.argsort(ratio)
    cw = np.cumsum(wgt[order])
    g_med = ratio[order][np.searchsorted(cw, 0.5 * cw[-1])]
    gamma, val = aa.aa_gamma_lp(A, f, "l1")
    assert val == pytest.approx(np.abs(a * g_med - f).sum(), rel=1e-10)
    assert gamma[0] == pytest.approx(g_med, rel=1e-8, abs=1e-10)


def test_linf_gamma_by_brute_force_over_pairs_for_one_column():
    """M = 1: max_i |a_i g - f_i| is convex piecewise linear in g; its minimum
    lies where two of the lines |a_i g - f_i| cross (pairs and signs)."""
    from oracle import aa
    A, f = _lp_data(30, 1, 2)
    a = A[:, 0]
    best = np.inf
    for i in range(len(a)):
        for j in range(i + 1, len(a)):
            for s in (1.0, -1.0):   # a_i g - f_i = s (a_j g - f_j)
                den = a[i] - s * a[j]
                if abs(den) < 1e-14:
                    continue
                g = (f[i] - s * f[j]) / den
                best = min(best, np.abs(a * g - f).max())
    _, val = aa.aa_gamma_lp(A, f, "linf")
    assert val == pytest.approx(best, rel=1e-10)


def test_l1_gamma_by_brute_force_over_interpolating_pairs():
    """M = 2: an l1 optimum interpolates two rows (a vertex of the LP): the
    minimum over all pairs of rows of the interpolant's objective."""
    from oracle import aa
    A, f = _lp_data(22, 2, 3)
    best = np.inf
    for i in range(len(f)):
        for j in range(i + 1, len(f)):
            B = A[[i, j]]
            if abs(np.linalg.det(B)) < 1e-12:
                continue
            g = np.linalg.solve(B, f[[i, j]])
            best = min(best, np.abs(A @ g - f).sum())
    _, val = aa.aa_gamma_lp(A, f, "l1")
    assert val == pytest.approx(best, rel=1e-10)


def test_linf_gamma_by_brute_force_over_levelled_triples():
    """M = 2: the minimax optimum levels three rows, s_i (A_i g - f_i) = t for
    signs s: the minimum over triples and signs of the levelled solutions'
    objective (t >= 0)."""
    import itertools
    from oracle import aa
    A, f = _lp_data(13, 2, 4)
    best = np.inf
    for tri in itertools.combinations(range(len(f)), 3):
        for sg in itertools.product((1.0, -1.0), repeat=3):
            K = np.array([[sg[q] * A[i, 0], sg[q] * A[i, 1], -1.0] for q, i in enumerate(tri)])
            if abs(np.linalg.det(K)) < 1e-12:
                continue
            sol = np.linalg.solve(K, np.array([sg[q] * f[i] for q, i in enumerate(tri)]))
            if sol[2] < 0:
                continue
            best = min(best, np.abs(A @ sol[:2] - f).max())
    _, val = aa.aa_gamma_lp(A, f, "linf")
    assert val == pytest.approx(best, rel=1e-10)


@pytest.mark.parametrize("norm", ["l1", "linf"])
def test_lp_gamma_weights_equal_scaled_rows(norm):
    """A weighted norm equals the plain norm of the rows scaled by the weights."""
    from oracle import aa
    A, f = _lp_data(200, 4, 5)
    w = np.exp(np.random.default_rng(6).uniform(-1.0, 1.0, len(f)))
    _, v1 = aa.aa_gamma_lp(A, f, norm, weights=w)
    _, v2 = aa.aa_gamma_lp(A * w[:, None], f * w, norm)
    assert v1 == pytest.approx(v2, rel=1e-10)


def test_host_lp_solver_matches_highs():
    """The library's host LP solver (aafwi_lp_min, no device call) against
    scipy's HiGHS on random bounded LPs, on degenerate ones (many rows through
    one vertex) and on the minimax fit of the l-infinity step."""
    from scipy.optimize import linprog
    from paper_2008_11778_gb300 import aafwi, build
    build.build()
    rng = np.random.default_rng(8)
    for nv, m in ((2, 7), (5, 40), (11, 400), (21, 300)):
        A = rng.standard_normal((m, nv))
        x0 = rng.standard_normal(nv)
        b = A @ x0 + rng.uniform(0.0, 1.0, m)
        box = np.vstack([np.eye(nv), -np.eye(nv)])
        A2, b2 = np.vstack([A, box]), np.r_[b, np.full(2 * nv, 50.0)]
        c = rng.standard_normal(nv)
        x, obj = aafwi.lp_min(A2, b2, c)
        ref = linprog(c, A_ub=A2, b_ub=b2, bounds=[(None, None)] * nv, method="highs")
        assert obj == pytest.approx(ref.fun, rel=1e-9, abs=1e-9)
        assert (A2 @ x <= b2 + 1e-8 * (1 + np.abs(b2))).all()
        # degenerate: 3 nv extra rows through the optimal vertex
        D = rng.standard_normal((3 * nv, nv))
        A3, b3 = np.vstack([A2, D]), np.r_[b2, D @ ref.x]
        x, obj = aafwi.lp_min(A3, b3, c)
        ref3 = linprog(c, A_ub=A3, b_ub=b3, bounds=[(None, None)] * nv, method="highs")
        assert obj == pytest.approx(ref3.fun, rel=1e-9, abs=1e-9)
    # minimax fit as the l-infinity step writes it
    from oracle import aa
    Af, f = _lp_data(300, 5, 9)
    one = np.ones((300, 1))
    A4 = np.block([[Af, -one], [-Af, -one]])
    x, obj = aafwi.lp_min(A4, np.r_[f, -f], np.r_[np.zeros(5), 1.0])
    assert obj == pytest.approx(aa.aa_gamma_lp(Af, f, "linf")[1], rel=1e-9)


def test_host_lp_solver_reports_an_unbounded_problem():
    from paper_2008_11778_gb300 import aafwi, build
    build.build()
    with pytest.raises(aafwi.AafwiError) as e:
        aafwi.lp_min(np.array([[1.0, 0.0]]), np.array([1.0]), np.array([0.0, 1.0]))   # min x2, x2 free
    assert e.value.code == 8
