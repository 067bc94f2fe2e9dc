"""Pins of the FP64 oracle's wave-equation operators (CPU only).

Each test checks the oracle against something other than itself: a closed
form, a textbook identity, an exact structural property or an adjoint /
finite-difference relation, so that a dropped term, a wrong sign or index, or
a transposed operand in oracle.c fails at least one of them.
"""
import math

import numpy as np
import pytest

from paper_2008_11778_gb300 import synth


# ---------------------------------------------------------------- stencil --

def test_laplacian_exact_on_polynomials_up_to_degree_9(orc):
    """8th-order central second difference is exact for degree <= 9 and its
    leading error on x^10 is the textbook -2 (4!)^2/10! h^8 u^(10) = -1152 h^8."""
    h = 0.1
    NZ, NX = 24, 30
    x = (np.arange(NX) - 15) * h
    z = (np.arange(NZ) - 12) * h
    for k in range(10):
        u = np.add.outer(0.5 * z ** k, x ** k)
        L = orc.laplacian(u, h, h)
        d2 = k * (k - 1) * x ** (k - 2) if k >= 2 else 0.0 * x
        d2z = 0.5 * k * (k - 1) * z ** (k - 2) if k >= 2 else 0.0 * z
        exact = np.add.outer(d2z, d2)
        assert np.abs(L - exact)[4:-4, 4:-4].max() < 1e-11 * max(1.0, np.abs(exact).max())
    u = np.tile(x ** 10, (NZ, 1))
    err = (orc.laplacian(u, h, h) - 90.0 * x ** 8)[4:-4, 4:-4]
    np.testing.assert_allclose(err, -1152.0 * h ** 8, rtol=1e-6)


def test_laplacian_zero_outside_and_anisotropic_spacing(orc):
    """A single unit spike: the stencil weights appear at +-1..4 along each
    axis scaled by 1/dz^2 and 1/dx^2 (Fornberg 8th-order weights)."""
    NZ, NX, dz, dx = 11, 13, 2.0, 3.0
    u = np.zeros((NZ, NX))
    u[5, 6] = 1.0
    L = orc.laplacian(u, dz, dx)
    w = [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]
    assert L[5, 6] == pytest.approx(w[0] / dz ** 2 + w[0] / dx ** 2, rel=1e-15)
    for k in range(1, 5):
        assert L[5 + k, 6] == pytest.approx(w[k] / dz ** 2, rel=1e-15)
        assert L[5, 6 - k] == pytest.approx(w[k] / dx ** 2, rel=1e-15)
    assert np.count_nonzero(L) == 17
    # spike at a corner: nothing wraps around
    u = np.zeros((NZ, NX))
    u[0, 0] = 1.0
    L = orc.laplacian(u, dz, dx)
    assert L[NZ - 1, 0] == 0.0 and L[0, NX - 1] == 0.0 and np.count_nonzero(L) == 9


# ------------------------------------------------------ extension, sponge --

def test_extension_adjoint_dot(orc):
    rng = np.random.default_rng(0)
    a = rng.standard_normal((7, 9))
    b = rng.standard_normal((7 + 6, 9 + 6))
    lhs = float((orc.extend(a, 3) * b).sum())
    rhs = float((a * orc.extend_adjoint(b, 3)).sum())
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)
    # E replicates the edge: corners of the pad equal the physical corners
    E = orc.extend(a, 3)
    assert (E[:3, :3] == a[0, 0]).all() and (E[-3:, -3:] == a[-1, -1]).all()
    assert (E[3:-3, 3:-3] == a).all()


def test_sponge_profile_is_one_inside_and_decays_outward(orc):
    G = orc.sponge(10, 12, 5)
    assert (G[5:-5, 5:-5] == 1.0).all()
    # monotone towards the outer edge, symmetric, below one in the pad
    assert (np.diff(G[5, :6]) > 0).all() and (np.diff(G[:6, 6]) > 0).all()
    np.testing.assert_array_equal(G, G[::-1, ::-1])
    assert G.max() == 1.0 and G.min() < 1.0


def test_sponge_is_the_product_of_the_axis_profiles(orc):
    """G = g(d_z) g(d_x) with g(d) = exp(-(0.015 d)^2), d = cells into the
    sponge: the reading of the non-reflecting boundary, written out."""
    nz, nx, nb = 7, 9, 6
    G = orc.sponge(nz, nx, nb)
    d = lambda i, n: max(nb - i, i - (nb + n - 1), 0)
    g = lambda dd: np.exp(-(0.015 * dd) ** 2)
    ref = np.array([[g(d(i, nz)) * g(d(j, nx)) for j in range(nx + 2 * nb)] for i in range(nz + 2 * nb)])
    np.testing.assert_allclose(G, ref, rtol=1e-15, atol=0)
    np.testing.assert_array_equal(G, np.outer(G[:, nb], G[nb, :]))   # separable, bitwise


def _point_geometry(n_phys, nb, h, dt, f, nt, offsets):
    cz = n_phys // 2
    g = synth.surface_geometry(n_phys, n_phys, nb, h, dt, f, nt, 1)
    g.src_iz[:] = cz
    g.src_ix[:] = cz
    g.rec_iz = np.full(len(offsets), cz, dtype=np.int32)
    g.rec_ix = np.array([cz + o for o in offsets], dtype=np.int32)
    g.rec_off = np.array([0, len(offsets)], dtype=np.int32)
    return g


def test_sponge_absorbs_boundary_reflections(orc):
    """Non-reflecting boundary (Sec. 2.2, eq. FWD): against a grid so large that
    no boundary echo returns within the window, the 20-cell sponge removes
    most of the echo that a bare grid edge produces."""
    def run(nb, pad):
        n = 101 + 2 * pad
        g = _point_geometry(n, nb, 10.0, 1e-3, 10.0, 800, [20])
        return orc.forward(g, np.full((n, n), 1 / 2000.0 ** 2))
    ref = run(0, 400)
    e_bare = np.linalg.norm(run(0, 0) - ref) / np.linalg.norm(ref)
    e_sponge = np.linalg.norm(run(20, 0) - ref) / np.linalg.norm(ref)
    assert e_bare > 0.5
    assert e_sponge < 0.1 * e_bare


# -------------------------------------------------------------- forward ----

def _green_ricker(r, c, f, times):
    """Homogeneous 2D Green's function of m u_tt - Lap u = w(t) delta(x),
    H(t - r/c) / (2 pi sqrt(t^2 - r^2/c^2)), convolved with the Ricker wavelet;
    the substitution tau = sqrt(t'^2 - r^2/c^2) removes the singularity."""
    from scipy import integrate
    t0 = 1.5 / f

    def w(t):
        a = (math.pi * f * (t - t0)) ** 2
        return (1 - 2 * a) * math.exp(-a) if t >= 0 else 0.0
    out = []
    for t in times:
        if t <= r / c:
            out.append(0.0)
            continue
        T = math.sqrt(t * t - r * r / (c * c))
        val, _ = integrate.quad(
            lambda tau: w(t - math.sqrt(tau * tau + r * r / (c * c))) / math.sqrt(tau * tau + r * r / (c * c)),
            0.0, T, limit=400)
        out.append(val / (2 * math.pi))
    return np.array(out)


@pytest.mark.slow
def test_forward_matches_2d_greens_function_and_converges_second_order(orc):
    """Amplitude (1/(dx dz) point source times W), timing (sample n = u^{n+1})
    and the leap-frog/8th-order scheme against the closed form; halving dt and
    h must cut the error ~4x (second order in time dominates)."""
    c, f, T = 2000.0, 10.0, 0.35
    errs = []
    for h, dt, n in ((5.0, 0.5e-3, 201), (2.5, 0.25e-3, 401)):
        offs_m = (100.0, 200.0)
        offs = [int(round(o / h)) for o in offs_m]
        nt = int(round(T / dt))
        g = _point_geometry(n, 20, h, dt, f, nt, offs)
        d = orc.forward(g, np.full((n, n), 1 / c ** 2)).reshape(nt, len(offs))
        times = (np.arange(nt) + 1) * dt
        e = []
        for j, o in enumerate(offs_m):
            a = _green_ricker(o, c, f, times)
            e.append(np.linalg.norm(d[:, j] - a) / np.linalg.norm(a))
        errs.append(np.array(e))
    assert (errs[0] < 2e-3).all()
    ratio = errs[0] / errs[1]
    assert ((ratio > 3.3) & (ratio < 4.7)).all(), ratio


def test_forward_causality_exact_zero(orc):
    """The cross-shaped radius-4 stencil moves support by at most 4 cells (l1)
    per step, so u^{n+1} at l1 distance D from the source is exactly 0 while
    4n < D, and becomes nonzero at n = D/4."""
    n = 61
    offs = [8, 16, 24]
    g = _point_geometry(n, 10, 10.0, 1e-3, 10.0, 12, offs)
    d = orc.forward(g, np.full((n, n), 1 / 2000.0 ** 2)).reshape(12, len(offs))
    for j, D in enumerate(offs):
        assert (d[: D // 4, j] == 0.0).all()
        assert d[D // 4, j] != 0.0


def test_forward_linear_in_source(orc):
    """Scaling the source scales the traces (bitwise for a factor 2), and the
    recurrence with a general source is additive in it."""
    p = synth.tiny()
    g = p.geom
    d1 = orc.forward(g, p.m_true)
    assert np.array_equal(orc.forward(g, p.m_true, amp=2.0), 2.0 * d1)
    rng = np.random.default_rng(11)
    NZ, NX, nt = 16, 19, 30
    W = (1e-3 ** 2) * rng.uniform(1500, 2500, (NZ, NX)) ** 2
    G = orc.sponge(NZ - 8, NX - 8, 4)
    riz, rix = np.array([3, 8, 12]), np.array([4, 9, 15])
    s1, s2 = rng.standard_normal((2, nt, NZ, NX))
    t12 = orc.propagate(W, G, 10.0, 10.0, s1 + s2, riz, rix)
    t1, t2 = (orc.propagate(W, G, 10.0, 10.0, s, riz, rix) for s in (s1, s2))
    np.testing.assert_allclose(t12, t1 + t2, rtol=0, atol=1e-12 * np.abs(t12).max())


def test_forward_is_the_propagator_with_a_point_ricker_source(orc):
    """The shot operator injects w(t_n)/(dx dz) at the source cell, w being the
    oracle's own Ricker samples: it equals the general recurrence driven by
    that point source, bitwise."""
    p = synth.small_problem()
    g = p.geom.subset([1])
    nt = int(g.nt[0])
    m = p.m_true
    d = orc.forward(g, m)
    mp = orc.extend(m, g.nb)
    W = g.dt ** 2 / mp
    G = orc.sponge(g.nz, g.nx, g.nb)
    s = np.zeros((nt,) + mp.shape)
    s[:, g.src_iz[0] + g.nb, g.src_ix[0] + g.nb] = orc.ricker(g.freq, g.dt, nt) * (1.0 / (g.dx * g.dz))
    tr = orc.propagate(W, G, g.dz, g.dx, s, g.rec_iz + g.nb, g.rec_ix + g.nb)
    assert np.array_equal(tr.ravel(), d)


def test_oracle_ricker_is_the_inputs_wavelet():
    """The oracle evaluates its source time function itself; the wavelet the
    input generator hands to the CUDA library (synth.ricker) must be the same
    samples, element by element."""
    import oracle as orc_mod
    for f, dt, nt in ((10.0, 1e-3, 600), (8.0, 1.5e-3, 2500), (15.0, 1e-3, 4000), (12.0, 0.8e-3, 6000)):
        a = orc_mod.ricker(f, dt, nt)
        b = synth.ricker(f, dt, nt)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)
        assert a.max() <= 1.0 and a.argmax() == int(round(1.5 / f / dt))


# -------------------------------------------------------------- adjoint ----

def test_propagator_dot_product(orc):
    """<P s, r> = <s, P^T r> for the forward recurrence and its transpose (eq. FWI_adj)."""
    rng = np.random.default_rng(1)
    NZ, NX, nt = 18, 23, 40
    W = (1e-3 ** 2) * rng.uniform(1500, 2500, (NZ, NX)) ** 2
    G = orc.sponge(NZ - 8, NX - 8, 4)
    riz = np.array([2, 5, 9, 9]); rix = np.array([3, 11, 4, 20])
    s = rng.standard_normal((nt, NZ, NX))
    r = rng.standard_normal((nt, len(riz)))
    lhs = float((orc.propagate(W, G, 10.0, 12.0, s, riz, rix) * r).sum())
    rhs = float((s * orc.propagate_adjoint(W, G, 10.0, 12.0, r, riz, rix)).sum())
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_fwi_gradient_central_differences(orc):
    """Central differences of J along a random direction converge at O(eps^2)
    to <grad J, dm> (exact discrete adjoint incl. sponge, E^T and the source)."""
    p = synth.small_problem()
    g = p.geom
    d_obs = orc.forward(g, p.m_true)
    m = p.m_start
    J, grad = orc.fwi_gradient(g, m, d_obs)
    rng = np.random.default_rng(3)
    dm = rng.standard_normal(m.shape) * m
    dd = float((grad * dm).sum())
    errs = []
    for eps in (1e-3, 1e-4):
        Jp, _ = orc.fwi_gradient(g, m + eps * dm, d_obs)
        Jm, _ = orc.fwi_gradient(g, m - eps * dm, d_obs)
        errs.append(abs((Jp - Jm) / (2 * eps) - dd) / abs(dd))
    assert errs[1] < 1e-7
    assert 50 < errs[0] / errs[1] < 200  # slope 2


def test_fwi_gradient_edge_cells_see_the_sponge(orc):
    """Perturbing one physical edge cell also changes the sponge cells that
    replicate it (extension E), so the gradient there must include the folded
    sponge contributions (E^T): checked by a one-cell difference quotient."""
    p = synth.small_problem()
    g = p.geom
    d_obs = orc.forward(g, p.m_true)
    m = p.m_start
    J, grad = orc.fwi_gradient(g, m, d_obs)
    for (iz, ix) in ((0, 0), (0, 17), (p.geom.nz - 1, 5)):
        e = np.zeros_like(m)
        e[iz, ix] = 1e-3 * m[iz, ix]
        Jp, _ = orc.fwi_gradient(g, m + e, d_obs)
        Jm, _ = orc.fwi_gradient(g, m - e, d_obs)
        fd = (Jp - Jm) / 2.0
        assert fd == pytest.approx(grad[iz, ix] * e[iz, ix], rel=1e-5)


# ----------------------------------------------------------------- Born ----

def test_born_dot_product(orc):
    """<L rho, d> = <rho, L^T d> (eqs. Born, FWI_adj)."""
    p = synth.small_problem()
    g = p.geom
    rng = np.random.default_rng(4)
    rho = rng.standard_normal(p.m_start.shape)
    d = rng.standard_normal(g.trace_count())
    lhs = float(orc.born_forward(g, p.m_true, rho) @ d)
    rhs = float((rho * orc.born_adjoint(g, p.m_true, d)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_born_is_the_derivative_of_forward(orc):
    """(F(m0(1+eps rho)) - F(m0(1-eps rho)))/(2 eps) -> L rho at O(eps^2)."""
    p = synth.small_problem()
    g = p.geom
    m0 = p.m_true
    rng = np.random.default_rng(5)
    rho = rng.standard_normal(m0.shape) * 0.1
    L = orc.born_forward(g, m0, rho)
    errs = []
    for eps in (1e-2, 1e-3):
        fd = (orc.forward(g, m0 * (1 + eps * rho)) - orc.forward(g, m0 * (1 - eps * rho))) / (2 * eps)
        errs.append(np.linalg.norm(fd - L) / np.linalg.norm(L))
    assert errs[1] < 1e-5
    assert 50 < errs[0] / errs[1] < 200


def test_lsrtm_objective_is_exactly_quadratic(orc):
    """J(rho + delta) = J(rho) + <grad, delta> + 1/2 ||L delta||^2 (eq. LSRTM)."""
    p = synth.small_problem()
    g = p.geom
    rng = np.random.default_rng(6)
    m0 = p.m_true
    rho = 0.05 * rng.standard_normal(m0.shape)
    delta = 0.05 * rng.standard_normal(m0.shape)
    d_obs = orc.born_forward(g, m0, 0.1 * rng.standard_normal(m0.shape))
    J, gr = orc.lsrtm_gradient(g, m0, rho, d_obs)
    J2, _ = orc.lsrtm_gradient(g, m0, rho + delta, d_obs)
    Ld = orc.born_forward(g, m0, delta)
    pred = J + float((gr * delta).sum()) + 0.5 * float(Ld @ Ld)
    assert J2 == pytest.approx(pred, rel=1e-11)


def test_fwi_gradient_equals_born_adjoint_of_residual(orc):
    """dJ/dm = (1/m) L^T r at the same model: the FWI imaging condition and the
    Born adjoint differ only by the factor dm = rho m."""
    p = synth.small_problem()
    g = p.geom
    d_obs = orc.forward(g, p.m_true)
    J, grad, r = orc.fwi_gradient(g, p.m_start, d_obs, want_resid=True)
    img = orc.born_adjoint(g, p.m_start, r)
    # E^T folds sponge cells of the same physical cell together; 1/m is uniform over them
    np.testing.assert_allclose(grad, img / p.m_start, rtol=1e-11, atol=1e-13 * np.abs(grad).max())
    assert J == pytest.approx(0.5 * float(r @ r), rel=1e-14)


def test_ricker_wavelet_properties():
    """The source time function (Sec. 4.1 names a Ricker wavelet by its centre
    frequency): unit peak at t0 = 1.5/f, symmetric about it, zero crossings at
    tau = +-1/(sqrt(2) pi f), zero mean, and an amplitude spectrum
    proportional to nu^2 exp(-nu^2/f^2), whose maximum sits at nu = f."""
    import math
    import oracle as orc_mod
    f, dt = 15.0, 1e-4
    n = 4000
    w = orc_mod.ricker(f, dt, n)
    t0 = 1.5 / f
    i0 = int(round(t0 / dt))
    assert abs(w[i0] - 1.0) < 1e-12 and w.argmax() == i0
    np.testing.assert_allclose(w[i0 - 500:i0], w[i0 + 500:i0:-1], atol=1e-12)
    tz = t0 + 1.0 / (math.sqrt(2.0) * math.pi * f)
    assert abs(synth.ricker(f, 1.0, 1, t0=-tz + t0)[0]) < 1e-12   # w at tau = tz - t0
    assert abs(orc_mod.ricker(f, tz, 2)[1]) < 1e-12                 # w(t0 + tz - t0) = w(tz)
    assert abs(w.sum() * dt) < 1e-6
    spec = np.abs(np.fft.rfft(w, 1 << 18)) * dt
    nu = np.fft.rfftfreq(1 << 18, dt)
    assert abs(nu[spec.argmax()] - f) < 0.05
    ref = nu ** 2 * np.exp(-(nu / f) ** 2)
    k = (nu > 2.0) & (nu < 60.0)
    ratio = spec[k] / ref[k]
    assert ratio.std() < 1e-3 * ratio.mean()
