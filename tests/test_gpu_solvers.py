"""The comparison solvers of Sec. 5 on the library's kernels against the
oracle: L-BFGS(M) with the Alg. 2 line search (quadratic objective and an
FWI problem with a data-sized residual) and restarted GMRES(M) (quadratic
system and the LSRTM normal equations L^T L x = L^T d)."""
import numpy as np
import pytest

from paper_2008_11778_gb300 import synth

pytestmark = pytest.mark.gpu
HIST_TOL = 1e-3


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_2008_11778_gb300 import aafwi, build
    build.build()
    aafwi.load()
    assert torch.cuda.is_available()
    return torch


def dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def quadratic(gpu, n, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, cond, n)) @ Q.T
    b = rng.standard_normal(n)
    return A, b, gpu.as_tensor(A, dtype=gpu.float64, device="cuda"), gpu.as_tensor(b, dtype=gpu.float64, device="cuda")


def test_dot_and_axpby(gpu):
    from paper_2008_11778_gb300 import aafwi
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(100003).astype(np.float32), rng.standard_normal(100003).astype(np.float32)
    X, Y = dev(gpu, x), dev(gpu, y)
    ref = float(np.dot(x.astype(np.float64), y.astype(np.float64)))
    assert abs(aafwi.dot(X, Y) - ref) <= 1e-12 * np.abs(x.astype(np.float64) * y).sum()
    aafwi.axpby(0.5, X, -2.0, Y)
    np.testing.assert_allclose(host(Y), 0.5 * x.astype(np.float64) - 2.0 * y, rtol=1e-6, atol=1e-6)
    Z = dev(gpu, y)
    aafwi.axpby_clip(0.5, X, -2.0, Z, -1.5, 2.0)          # the line-search bound constraint
    np.testing.assert_allclose(host(Z), np.clip(0.5 * x.astype(np.float64) - 2.0 * y, -1.5, 2.0), rtol=1e-6, atol=1e-6)
    W = dev(gpu, y)
    aafwi.axpby_clip(0.5, X, -2.0, W, 1.0, 1.0)           # lo >= hi: no clip
    assert gpu.equal(W, Y)


@pytest.mark.parametrize("curvature", [False, True], ids=["armijo", "wolfe"])
def test_lbfgs_quadratic_history_matches_oracle(gpu, curvature):
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import solve
    n = 300
    A, b, At, bt = quadratic(gpu, n, 200.0, 5)

    def grad_fn(x, g_out, reuse):
        xd = x.double()
        g_out.copy_((At @ xd - bt).float())
        return float(0.5 * xd @ (At @ xd) - bt @ xd)

    def misfit_fn(x):
        xd = x.double()
        return float(0.5 * xd @ (At @ xd) - bt @ xd)

    out = solve.lbfgs_fwi(None, None, gpu.zeros(n, device="cuda"), M=5, iters=25, eta=1.0 / 200.0,
                          grad_fn=grad_fn, misfit_fn=misfit_fn, curvature=curvature)

    def ogf(x):
        x32 = x.astype(np.float32).astype(np.float64)
        return 0.5 * x32 @ A @ x32 - b @ x32, (A @ x32 - b).astype(np.float32).astype(np.float64)
    ref = oaa.lbfgs(ogf, np.zeros(n), M=5, eta=1.0 / 200.0, iters=25, misfit_fn=lambda x: ogf(x)[0],
                    curvature=curvature)
    assert out["lam"] == ref["lam"]
    Jstar = -0.5 * b @ np.linalg.solve(A, b)
    assert rel(np.array(out["J"]) - Jstar, np.array(ref["J"]) - Jstar) < HIST_TOL
    assert rel(host(out["p"]), ref["p"][-1]) < 1e-4


def test_lbfgs_fwi_history_large_residual(gpu, orc):
    """L-BFGS(5) with the weak-Wolfe search, 8 iterations, on the data-sized-
    residual problem of the AA history test: the misfit history matches the
    oracle's to the 1e-3 target."""
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import aafwi, solve
    p = synth.small_problem(nz=48, nx=120, nb=12, nt=300, S=3)
    g = p.geom
    d_obs = orc.forward(g, p.m_true).astype(np.float32)
    lo, hi = p.m_bounds
    plan = aafwi.Plan(g, max(float(p.c_true.max()), p.c_bounds[1]))
    out = solve.lbfgs_fwi(plan, dev(gpu, d_obs), dev(gpu, p.m_start), M=5, iters=8, eta_factor=1e-3,
                          bounds=(lo, hi), curvature=True)
    ref = oaa.lbfgs(lambda m: orc.fwi_gradient(g, m.astype(np.float32), d_obs),
                    p.m_start.astype(np.float32).astype(np.float64), M=5, eta=out["eta"], iters=8,
                    bounds=(lo, hi), curvature=True)
    assert out["lam"] == ref["lam"]
    assert rel(out["J"], ref["J"]) < HIST_TOL
    assert ref["J"][-1] < 0.9 * ref["J"][0]


def test_gmres_quadratic_matches_oracle(gpu):
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import solve
    n = 300
    A, b, At, bt = quadratic(gpu, n, 50.0, 6)

    def residual_fn(x, out):
        out.copy_((At @ x.double() - bt).float())

    x0 = np.zeros(n, dtype=np.float32)
    out = solve.gmres_restarted(residual_fn, dev(gpu, x0), M=4, iters=16)
    xs, res = oaa.gmres_restarted(lambda v: A @ v, b, x0.astype(np.float64), M=4, iters=16)
    assert rel(out["res"], res) < HIST_TOL
    assert rel(host(out["x"]), xs[-1]) < 1e-4
    assert out["applications"] == 1 + 16 + 4          # b, one per step, one per restart


def test_gmres_lsrtm_normal_equations_vs_oracle(gpu, orc):
    """GMRES(3) on L^T L x = L^T d (eq. LSRTM3), 6 steps from the RTM image,
    with the library's LSRTM gradient as the residual map, against the oracle
    GMRES on the oracle's Born operators."""
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import aafwi, solve
    p = synth.small_problem(nz=40, nx=64, nb=8, nt=180, S=2)
    g = p.geom
    rng = np.random.default_rng(7)
    m0 = p.m_true.astype(np.float32)
    rho_true = (0.1 * rng.standard_normal(m0.shape)).astype(np.float32)
    d = orc.born_forward(g, m0, rho_true).astype(np.float32)
    plan = aafwi.Plan(g, float(p.c_true.max()))
    M0, D = dev(gpu, m0), dev(gpu, d)
    rtm = gpu.empty_like(M0)
    plan.born_adjoint(M0, D, rtm)
    x0 = host(rtm)

    def residual_fn(x, out):
        plan.adjoint_gradient(aafwi.MODE_LSRTM, M0, x, D, out, sync=False)

    out = solve.gmres_restarted(residual_fn, rtm, M=3, iters=6)
    b = orc.born_adjoint(g, m0, d)
    xs, res = oaa.gmres_restarted(lambda v: orc.born_adjoint(g, m0, orc.born_forward(g, m0, v)), b,
                                  x0, M=3, iters=6)
    assert rel(out["res"], res) < HIST_TOL
    assert rel(host(out["x"]), xs[-1]) < 1e-3
    assert res[-1] < 0.5 * res[0]


@pytest.mark.parametrize("beta", [0.5, 0.8])
def test_damped_aa_quadratic_history_matches_oracle(gpu, beta):
    """Alg. 2 with the damped AA point (Alg. 1 eq. AAupdate0, beta < 1) on a
    quadratic: line-search decisions, misfit gap and iterate against the oracle."""
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import solve
    n = 300
    A, b, At, bt = quadratic(gpu, n, 200.0, 8)

    def grad_fn(x, g_out, reuse):
        xd = x.double()
        g_out.copy_((At @ xd - bt).float())
        return float(0.5 * xd @ (At @ xd) - bt @ xd)

    def misfit_fn(x):
        xd = x.double()
        return float(0.5 * xd @ (At @ xd) - bt @ xd)

    out = solve.aa_fwi(None, None, gpu.zeros(n, device="cuda"), M=5, iters=20, eta=1.0 / 200.0,
                       grad_fn=grad_fn, misfit_fn=misfit_fn, beta=beta)

    def ogf(x):
        x32 = x.astype(np.float32).astype(np.float64)
        return 0.5 * x32 @ A @ x32 - b @ x32, (A @ x32 - b).astype(np.float32).astype(np.float64)
    ref = oaa.aa_gd(ogf, np.zeros(n), M=5, eta=1.0 / 200.0, iters=20, misfit_fn=lambda x: ogf(x)[0], beta=beta)
    assert out["lam"] == ref["lam"]
    Jstar = -0.5 * b @ np.linalg.solve(A, b)
    assert rel(np.array(out["J"]) - Jstar, np.array(ref["J"]) - Jstar) < HIST_TOL
    assert rel(host(out["p"]), ref["p"][-1]) < 1e-4


def test_weighted_aa_quadratic_history_matches_oracle(gpu):
    """Alg. 2 with a weighted l2 norm in the AA least squares (diagonal
    weights 0.1..10) against the oracle."""
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import solve
    n = 300
    A, b, At, bt = quadratic(gpu, n, 200.0, 9)
    w = np.exp(np.random.default_rng(10).uniform(np.log(0.1), np.log(10.0), n)).astype(np.float32)

    def grad_fn(x, g_out, reuse):
        xd = x.double()
        g_out.copy_((At @ xd - bt).float())
        return float(0.5 * xd @ (At @ xd) - bt @ xd)

    def misfit_fn(x):
        xd = x.double()
        return float(0.5 * xd @ (At @ xd) - bt @ xd)

    out = solve.aa_fwi(None, None, gpu.zeros(n, device="cuda"), M=5, iters=20, eta=1.0 / 200.0,
                       grad_fn=grad_fn, misfit_fn=misfit_fn, weights=dev(gpu, w))

    def ogf(x):
        x32 = x.astype(np.float32).astype(np.float64)
        return 0.5 * x32 @ A @ x32 - b @ x32, (A @ x32 - b).astype(np.float32).astype(np.float64)
    ref = oaa.aa_gd(ogf, np.zeros(n), M=5, eta=1.0 / 200.0, iters=20, misfit_fn=lambda x: ogf(x)[0],
                    weights=w.astype(np.float64))
    assert out["lam"] == ref["lam"]
    Jstar = -0.5 * b @ np.linalg.solve(A, b)
    assert rel(np.array(out["J"]) - Jstar, np.array(ref["J"]) - Jstar) < HIST_TOL
    assert rel(host(out["p"]), ref["p"][-1]) < 1e-4


def test_noisy_data_aa_fwi_history_matches_oracle(gpu, orc):
    """The noisy-data experiment (Sec. 4.2): observed data with mean-zero
    uniform noise at SNR 0.55 dB, Alg. 2 with AA(5) for 10 iterations on the
    GPU against the oracle's run on the same noisy data (misfit history and
    line-search decisions at the 1e-3 target)."""
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import aafwi, solve
    p = synth.small_problem(nz=48, nx=120, nb=12, nt=300, S=3)
    g = p.geom
    clean = orc.forward(g, p.m_true)
    noise = synth.uniform_noise(clean, 0.55, seed=4 * 1000 + 2008)
    snr = 10.0 * np.log10(np.mean(clean ** 2) / np.mean(noise ** 2))
    assert abs(snr - 0.55) < 0.05 and abs(noise.mean()) < 0.05 * noise.std()
    d_obs = (clean + noise).astype(np.float32)
    lo, hi = p.m_bounds
    plan = aafwi.Plan(g, p.c_bounds[1])
    out = solve.aa_fwi(plan, dev(gpu, d_obs), dev(gpu, p.m_start), M=5, iters=10, eta_factor=1e-3,
                       bounds=(lo, hi))
    ref = oaa.aa_gd(lambda m: orc.fwi_gradient(g, m.astype(np.float32), d_obs),
                    p.m_start.astype(np.float32).astype(np.float64), M=5, eta=out["eta"], iters=10,
                    bounds=(lo, hi),
                    misfit_fn=lambda m: 0.5 * float(np.sum((orc.forward(g, m.astype(np.float32)) - d_obs) ** 2)))
    assert out["lam"] == ref["lam"]
    assert rel(out["J"], ref["J"]) < HIST_TOL
    assert ref["J"][-1] < ref["J"][0]
    plan.close()


@pytest.mark.parametrize("norm, weighted", [("l1", False), ("linf", False), ("l1", True), ("linf", True)],
                         ids=["l1", "linf", "l1-weighted", "linf-weighted"])
def test_aa_lp_step_matches_oracle(gpu, norm, weighted):
    """AA with the l1 / l-infinity norm in the optimisation step (Sec. 2.1):
    over a sliding window the GPU rounds reach the oracle's LP optimum (the
    optimal value is unique; gamma need not be), the GPU gamma attains it,
    and the AA point is formed from that gamma."""
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import aafwi
    rng = np.random.default_rng(31 if norm == "l1" else 32)
    n, M, eta = 6001, 4, 0.03
    A = rng.standard_normal((40, n)) / 20.0
    w = np.exp(rng.uniform(-1.0, 1.0, n)).astype(np.float32) if weighted else None
    st = aafwi.AA(n, M, eta)
    st.set_norm(aafwi.NORM_L1 if norm == "l1" else aafwi.NORM_LINF)
    if weighted:
        st.set_weights(dev(gpu, w))
    pt, pb = gpu.empty(n, device="cuda"), gpu.empty(n, device="cuda")
    x = rng.standard_normal(n).astype(np.float32)
    ps, gs = [], []
    w64 = None if w is None else w.astype(np.float64)
    for k in range(8):
        gk = (A.T @ (A @ x) + 0.1 * x + 0.05 * rng.laplace(size=n)).astype(np.float32)
        ps.append(x.astype(np.float64))
        gs.append(gk.astype(np.float64))
        gam, Mk = st.step(dev(gpu, x), dev(gpu, gk), pt, pb, want_gamma=True)
        P, G = ps[-(M + 1):], gs[-(M + 1):]
        ref_bar, ref_tilde, ref_gam, ref_Mk = oaa.anderson_point(P, G, eta, weights=w64, norm=norm)
        assert Mk == ref_Mk == min(M, k)
        if Mk:
            dG = np.stack([G[i + 1] - G[i] for i in range(len(G) - 1)], axis=1)[:, -Mk:]
            _, opt = oaa.aa_gamma_lp(dG, G[-1], norm, w64)
            wt = np.ones(n) if w64 is None else w64
            r = np.abs(wt * (dG @ gam - G[-1]))
            val = r.max() if norm == "linf" else r.sum()
            info = st.lp_info()
            assert val == pytest.approx(opt, rel=1e-7)                 # gamma attains the optimum
            assert info["objective"] == pytest.approx(val, rel=1e-9)
            assert info["lower_bound"] <= info["objective"] * (1 + 1e-9)
            # the AA point of this gamma (eq. AA2_update), formed in FP64 here
            tilde = P[-1] - eta * G[-1] - sum(g * ((P[-Mk + i] - eta * G[-Mk + i]) - (P[-Mk - 1 + i] - eta * G[-Mk - 1 + i]))
                                              for i, g in enumerate(gam))
            assert rel(host(pt), tilde) < 1e-6
        assert rel(host(pb), ref_bar) < 1e-6
        x = (0.5 * ref_tilde + 0.5 * ref_bar + 0.01 * rng.standard_normal(n)).astype(np.float32)
    st.close()


@pytest.mark.parametrize("norm", ["l1", "linf"])
def test_aa_lp_quadratic_history_matches_oracle(gpu, norm):
    """Alg. 2 with the l1 / l-infinity AA step on a quadratic: line-search
    decisions, misfit gap and iterate against the oracle's Alg. 2."""
    from oracle import aa as oaa
    from paper_2008_11778_gb300 import aafwi, solve
    n = 300
    A, b, At, bt = quadratic(gpu, n, 200.0, 12)

    def grad_fn(x, g_out, reuse):
        xd = x.double()
        g_out.copy_((At @ xd - bt).float())
        return float(0.5 * xd @ (At @ xd) - bt @ xd)

    def misfit_fn(x):
        xd = x.double()
        return float(0.5 * xd @ (At @ xd) - bt @ xd)

    out = solve.aa_fwi(None, None, gpu.zeros(n, device="cuda"), M=5, iters=20, eta=1.0 / 200.0,
                       grad_fn=grad_fn, misfit_fn=misfit_fn,
                       norm=aafwi.NORM_L1 if norm == "l1" else aafwi.NORM_LINF)

    def ogf(x):
        x32 = x.astype(np.float32).astype(np.float64)
        return 0.5 * x32 @ A @ x32 - b @ x32, (A @ x32 - b).astype(np.float32).astype(np.float64)
    ref = oaa.aa_gd(ogf, np.zeros(n), M=5, eta=1.0 / 200.0, iters=20, misfit_fn=lambda x: ogf(x)[0], norm=norm)
    assert out["lam"] == ref["lam"]
    Jstar = -0.5 * b @ np.linalg.solve(A, b)
    assert rel(np.array(out["J"]) - Jstar, np.array(ref["J"]) - Jstar) < HIST_TOL
    assert (np.array(ref["J"]) - Jstar)[-1] < 0.5 * (np.array(ref["J"]) - Jstar)[1]
