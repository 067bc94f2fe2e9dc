"""Seeded synthetic inputs: velocity models, acquisition geometry, wavelets.

This module holds no arithmetic of the inversion method.  It only draws the
inputs that both the CUDA library and its FP64 checker consume: it imports
numpy (and scipy for the Gaussian smoothing of start models) and nothing else
from this package.

The paper's Marmousi model and data are not available; these seeded models
stand in for them with the shapes, sizes and structure of each workload:

  tiny      101 x 51, dx 10 m, two layers (1500/2000 m/s, interface at
            row 25) + Gaussian anomaly (+200 m/s, radius 8 cells); 3 surface
            shots, 101 receivers, Ricker 10 Hz, dt 1 ms, 600 steps.
  batched   400 x 150, dx 20 m, 12 dipping layers 1500-4500 m/s cut by two
            60-degree normal faults; start = Gaussian-smoothed (sigma 10);
            32 shots, spreads of 60-400 receivers, Ricker 8 Hz, dt 1.5 ms,
            2500 steps.
  lsrtm     737 x 240, dx 12.5 m, background 1500-4700 m/s linear in depth,
            40 faulted one-cell reflectors with reflectivity in [-0.1, 0.1];
            64 shots, 369 receivers, Ricker 15 Hz, dt 1 ms, 4000 steps.
  large     2001 x 601, dx 10 m, layered-faulted 1500-5500 m/s with three
            +800 m/s elliptic lenses; 200 shots with uneven apertures,
            Ricker 12 Hz, dt 0.8 ms, 6000 steps.
  learned   256 x 96, dx 20 m models from the batched generator (training),
            16 shots, Ricker 10 Hz, dt 1.5 ms, 1500 steps; held-out 400 x 150
            evaluation models of the same generator, 2500 steps.

Sources and receivers sit one cell below the top of the physical grid; shot
s of S is at column round((s + 1/2) nx / S).  Seeds are 1000*id + 2008.
"""
from dataclasses import dataclass, field
import math

import numpy as np

NB_DEFAULT = 20


def ricker(f, dt, nt, t0=None):
    """Ricker wavelet w(t) = (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2),
    tau = t - t0, t0 = 1.5/f, sampled at t_n = n dt (float64)."""
    if t0 is None:
        t0 = 1.5 / f
    t = np.arange(nt, dtype=np.float64) * dt
    a = (math.pi * f * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


@dataclass
class Geometry:
    nz: int
    nx: int
    nb: int
    dz: float
    dx: float
    dt: float
    src_iz: np.ndarray
    src_ix: np.ndarray
    nt: np.ndarray
    rec_off: np.ndarray
    rec_iz: np.ndarray
    rec_ix: np.ndarray
    wavelet: np.ndarray
    freq: float = 0.0

    @property
    def S(self):
        return len(self.src_iz)

    @property
    def NZ(self):
        return self.nz + 2 * self.nb

    @property
    def NX(self):
        return self.nx + 2 * self.nb

    @property
    def nrec(self):
        return np.diff(self.rec_off)

    def trace_offsets(self):
        return np.concatenate([[0], np.cumsum(self.nt.astype(np.int64) * self.nrec)])

    def trace_count(self):
        return int(self.trace_offsets()[-1])

    def updates_per_pass(self):
        """Grid-point updates of one pass over every shot: sum_s nt_s * NZ * NX."""
        return int(self.nt.astype(np.int64).sum()) * self.NZ * self.NX

    def subset(self, shots):
        """Geometry restricted to the listed shots (same grid and wavelet)."""
        shots = list(shots)
        off = []
        iz, ix = [], []
        o = 0
        for s in shots:
            a, b = self.rec_off[s], self.rec_off[s + 1]
            off.append(o)
            iz.append(self.rec_iz[a:b])
            ix.append(self.rec_ix[a:b])
            o += b - a
        off.append(o)
        return Geometry(self.nz, self.nx, self.nb, self.dz, self.dx, self.dt,
                        self.src_iz[shots].copy(), self.src_ix[shots].copy(),
                        self.nt[shots].copy(), np.array(off, dtype=np.int32),
                        np.concatenate(iz).astype(np.int32), np.concatenate(ix).astype(np.int32),
                        self.wavelet.copy(), self.freq)

    def with_nt(self, nt):
        g = self.subset(range(self.S))
        g.nt = np.minimum(g.nt, nt).astype(np.int32)
        return g


@dataclass
class Problem:
    name: str
    geom: Geometry
    c_true: np.ndarray           # [nz, nx] velocity (m/s), float64
    c_start: np.ndarray          # [nz, nx] start velocity (m/s)
    M: int = 5
    iters: int = 10
    c_bounds: tuple = (0.0, 0.0)  # velocity clip applied after each update
    extra: dict = field(default_factory=dict)

    @property
    def m_true(self):
        return 1.0 / self.c_true ** 2

    @property
    def m_start(self):
        return 1.0 / self.c_start ** 2

    @property
    def m_bounds(self):
        """Velocity clip mapped to m = 1/c^2: (lo, hi) with lo = 1/c_hi^2."""
        lo, hi = self.c_bounds
        return 1.0 / hi ** 2, 1.0 / lo ** 2


def surface_geometry(nz, nx, nb, dx, dt, f, nt, S, spreads=None, nt_per_shot=None,
                     rec_step=1, depth=1):
    """S shots at depth ``depth`` (cells), column round((s+1/2) nx/S).

    spreads: None -> every ``rec_step``-th column of the grid for all shots;
    otherwise an int array of spread lengths (receivers at every column)
    centred on each source and clipped to the grid.
    """
    src_ix = np.array([int(round((s + 0.5) * nx / S)) for s in range(S)], dtype=np.int32)
    src_ix = np.clip(src_ix, 0, nx - 1)
    src_iz = np.full(S, depth, dtype=np.int32)
    rec_off, rec_iz, rec_ix = [0], [], []
    for s in range(S):
        if spreads is None:
            cols = np.arange(0, nx, rec_step)
        else:
            L = int(spreads[s])
            a = max(0, int(src_ix[s]) - L // 2)
            b = min(nx, a + L)
            a = max(0, b - L)
            cols = np.arange(a, b)
        rec_ix.append(cols)
        rec_iz.append(np.full(len(cols), depth))
        rec_off.append(rec_off[-1] + len(cols))
    ntv = np.full(S, nt, dtype=np.int32) if nt_per_shot is None else np.asarray(nt_per_shot, dtype=np.int32)
    return Geometry(nz, nx, nb, float(dx), float(dx), float(dt), src_iz, src_ix, ntv,
                    np.array(rec_off, dtype=np.int32),
                    np.concatenate(rec_iz).astype(np.int32),
                    np.concatenate(rec_ix).astype(np.int32),
                    ricker(f, dt, int(ntv.max())), float(f))


def layered_faulted(nz, nx, nlayers, vmin, vmax, nfaults, rng, max_dip_deg=8.0,
                    throw=(5, 15), jitter=100.0):
    """Dipping layers (velocities evenly spaced vmin..vmax plus U(-jitter, jitter),
    thicknesses from a Dirichlet split of nz), cut by 60-degree normal faults."""
    vel = np.linspace(vmin, vmax, nlayers) + rng.uniform(-jitter, jitter, nlayers)
    vel = np.clip(vel, vmin, vmax)
    thick = rng.dirichlet(np.full(nlayers, 2.0)) * nz
    tops = np.concatenate([[0.0], np.cumsum(thick)[:-1]])
    dip = math.tan(math.radians(rng.uniform(-max_dip_deg, max_dip_deg)))
    zz, xx = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(nx, dtype=np.float64),
                         indexing="ij")
    zs = zz.copy()
    for _ in range(nfaults):
        x0 = rng.uniform(0.2 * nx, 0.8 * nx)
        t = rng.uniform(throw[0], throw[1])
        hanging = xx > x0 + zz / math.tan(math.radians(60.0))
        zs = np.where(hanging, zs - t, zs)
    zref = zs - dip * (xx - nx / 2.0)
    idx = np.searchsorted(tops, zref, side="right") - 1
    idx = np.clip(idx, 0, nlayers - 1)
    return vel[idx]


def _smooth(c, sigma):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(c, sigma, mode="nearest")


def tiny(nb=NB_DEFAULT):
    """Two-layer model with a Gaussian anomaly; 3 shots, 101 receivers."""
    nz, nx = 51, 101
    c0 = np.where(np.arange(nz)[:, None] < 25, 1500.0, 2000.0) * np.ones((1, nx))
    zz, xx = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    r2 = (zz - 38.0) ** 2 + (xx - 50.0) ** 2
    c_true = c0 + 200.0 * np.exp(-r2 / 8.0 ** 2)
    g = surface_geometry(nz, nx, nb, 10.0, 1e-3, 10.0, 600, 3)
    return Problem("tiny-101x51", g, c_true, c0.copy(), M=5, iters=10,
                   c_bounds=(0.8 * 1500.0, 1.2 * 2200.0))


def batched(nb=NB_DEFAULT, uneven_nt=False, seed=1 * 1000 + 2008):
    """12 dipping layers, 2 normal faults; 32 shots with uneven spreads."""
    rng = np.random.default_rng(seed)
    nz, nx = 150, 400
    c_true = layered_faulted(nz, nx, 12, 1500.0, 4500.0, 2, rng)
    c_start = _smooth(c_true, 10.0)
    spreads = rng.integers(60, 401, size=32)
    ntv = rng.integers(1500, 2501, size=32) if uneven_nt else None
    g = surface_geometry(nz, nx, nb, 20.0, 1.5e-3, 8.0, 2500, 32, spreads=spreads,
                         nt_per_shot=ntv)
    return Problem("batched-400x150", g, c_true, c_start, M=10, iters=30,
                   c_bounds=(0.8 * c_true.min(), 1.2 * c_true.max()))


def lsrtm(nb=NB_DEFAULT, seed=2 * 1000 + 2008):
    """Linear-in-depth background and 40 faulted one-cell reflectors."""
    rng = np.random.default_rng(seed)
    nz, nx = 240, 737
    c_bg = (1500.0 + 3200.0 * np.arange(nz) / (nz - 1))[:, None] * np.ones((1, nx))
    rho = np.zeros((nz, nx))
    faults = [(rng.uniform(0.15 * nx, 0.85 * nx), rng.uniform(3, 12)) for _ in range(3)]
    xs = np.arange(nx, dtype=np.float64)
    for _ in range(40):
        z0 = rng.uniform(10, nz - 10)
        slope = math.tan(math.radians(rng.uniform(-15.0, 15.0)))
        amp = rng.uniform(-0.1, 0.1)
        z = z0 + slope * (xs - nx / 2.0)
        for x0, t in faults:
            z = np.where(xs > x0, z + t, z)
        zi = np.rint(z).astype(int)
        ok = (zi >= 0) & (zi < nz)
        rho[zi[ok], np.nonzero(ok)[0]] = amp
    g = surface_geometry(nz, nx, nb, 12.5, 1e-3, 15.0, 4000, 64, rec_step=2)
    p = Problem("lsrtm-737x240", g, c_bg, c_bg.copy(), M=5, iters=20)
    p.extra["rho_true"] = rho
    return p


def large(nb=NB_DEFAULT, seed=3 * 1000 + 2008):
    """Layered-faulted 1500-5500 m/s with three high-velocity lenses; 200 shots."""
    rng = np.random.default_rng(seed)
    nz, nx = 601, 2001
    c = layered_faulted(nz, nx, 16, 1500.0, 5500.0, 3, rng)
    zz, xx = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    for _ in range(3):
        cz, cx = rng.uniform(0.3 * nz, 0.8 * nz), rng.uniform(0.1 * nx, 0.9 * nx)
        az, ax = rng.uniform(20, 60, size=2)
        inside = ((zz - cz) / az) ** 2 + ((xx - cx) / ax) ** 2 <= 1.0
        c = np.where(inside, np.minimum(c + 800.0, 5500.0), c)
    spreads = rng.integers(200, 2002, size=200)
    g = surface_geometry(nz, nx, nb, 10.0, 0.8e-3, 12.0, 6000, 200, spreads=spreads)
    return Problem("large-2001x601", g, c, _smooth(c, 10.0), M=10, iters=30,
                   c_bounds=(0.8 * c.min(), 1.2 * c.max()))


def learned_model(seed, nz=96, nx=256, nb=NB_DEFAULT):
    """One training model of the learned-preconditioner set (batched generator
    rescaled to 256 x 96), 16 shots, Ricker 10 Hz, dt 1.5 ms, 1500 steps."""
    rng = np.random.default_rng(seed)
    c_true = layered_faulted(nz, nx, 12, 1500.0, 4500.0, 2, rng, throw=(3, 9))
    c_start = _smooth(c_true, 6.0)
    g = surface_geometry(nz, nx, nb, 20.0, 1.5e-3, 10.0, 1500, 16)
    return Problem("learned-%dx%d-%d" % (nx, nz, seed), g, c_true, c_start, M=10, iters=30,
                   c_bounds=(0.8 * c_true.min(), 1.2 * c_true.max()))


def learned_eval_model(seed, nz=150, nx=400, nb=NB_DEFAULT):
    """A held-out evaluation model of the learned preconditioner: 400 x 150,
    the training generator's structure and acquisition (dx 20 m, 16 shots,
    Ricker 10 Hz, dt 1.5 ms) with a record long enough for the wider spread
    (2500 steps)."""
    rng = np.random.default_rng(seed)
    c_true = layered_faulted(nz, nx, 12, 1500.0, 4500.0, 2, rng, throw=(3, 9))
    c_start = _smooth(c_true, 6.0)
    g = surface_geometry(nz, nx, nb, 20.0, 1.5e-3, 10.0, 2500, 16)
    return Problem("learned-eval-%dx%d-%d" % (nx, nz, seed), g, c_true, c_start, M=10, iters=30,
                   c_bounds=(0.8 * c_true.min(), 1.2 * c_true.max()))


def small_problem(nz=30, nx=40, nb=8, nt=160, S=2, dx=10.0, dt=1e-3, f=15.0, seed=7):
    """A few-second problem for gradient/adjoint checks on tiny grids: a
    smooth random model (1800-2400 m/s) with surface shots and receivers."""
    rng = np.random.default_rng(seed)
    zz, xx = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    c = 1800.0 + 300.0 * zz / max(nz - 1, 1)
    for _ in range(3):
        cz, cx = rng.uniform(0, nz), rng.uniform(0, nx)
        c = c + rng.uniform(-150, 150) * np.exp(-((zz - cz) ** 2 + (xx - cx) ** 2) / 30.0)
    g = surface_geometry(nz, nx, nb, dx, dt, f, nt, S)
    return Problem("small-%dx%d" % (nx, nz), g, c, np.full_like(c, c.mean()), M=5, iters=10,
                   c_bounds=(1500.0, 3000.0))


def uniform_noise(d, snr_db, seed):
    """Mean-zero uniform noise for traces d at the given signal-to-noise ratio
    (10 log10 of mean signal power over noise power): U(-a, a) with
    a^2 / 3 = mean(d^2) / 10^(snr_db / 10).  Seeded; returns the noise only."""
    d = np.asarray(d, dtype=np.float64)
    p_noise = float(np.mean(d * d)) / 10.0 ** (snr_db / 10.0)
    a = np.sqrt(3.0 * p_noise)
    return np.random.default_rng(seed).uniform(-a, a, d.shape)
