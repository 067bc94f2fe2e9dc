"""FP64 CPU oracle for the Anderson-accelerated FWI / LSRTM hot path.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product package.  It shares no code
with the CUDA library; the two meet only through the seeded input generators.

Wave-equation operators (forward F, FWI gradient, Born L and L^T) live in
oracle.c and are reached through ctypes; the Anderson-acceleration optimiser
(Alg. 1 / Alg. 2) and full-memory GMRES are in ``oracle.aa``.

A geometry object is anything with the attributes
  nz, nx, nb, dz, dx, dt        physical grid, sponge width, spacing, time step
  src_iz, src_ix                [S] int physical source cells
  nt                            [S] int record length per shot
  rec_off, rec_iz, rec_ix       CSR receivers per shot (physical cells)
  freq                          Ricker centre frequency f (Hz)
The source time function is the oracle's own: oracle.c evaluates the Ricker
wavelet w(t_n), t_n = n dt, with delay 1.5/f (``ricker`` returns its samples).
Traces are a flat float64 array: shot s at offset sum_{q<s} nt_q*nrec_q,
time-major [nt_s][nrec_s].
"""
import ctypes
import numpy as np

from .build import build_oracle

_lib = None


class _Geom(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int), ("nx", ctypes.c_int), ("nb", ctypes.c_int),
                ("dz", ctypes.c_double), ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("S", ctypes.c_int),
                ("src_iz", ctypes.c_void_p), ("src_ix", ctypes.c_void_p),
                ("nt", ctypes.c_void_p), ("rec_off", ctypes.c_void_p),
                ("rec_iz", ctypes.c_void_p), ("rec_ix", ctypes.c_void_p),
                ("freq", ctypes.c_double), ("amp", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.og_laplacian.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P]
        L.og_sponge.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
        L.og_extend.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]
        L.og_extend_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]
        L.og_propagate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   P, P, ctypes.c_int, P, ctypes.c_int, P, P, P]
        L.og_propagate_adjoint.argtypes = L.og_propagate.argtypes
        L.og_trace_count.argtypes = [P]
        L.og_trace_count.restype = ctypes.c_size_t
        L.og_forward.argtypes = [P, P, P]
        L.og_fwi_gradient.argtypes = [P, P, P, P, P]
        L.og_fwi_gradient.restype = ctypes.c_double
        L.og_born_forward.argtypes = [P, P, P, P]
        L.og_born_adjoint.argtypes = [P, P, P, P]
        L.og_num_threads.restype = ctypes.c_int
        L.og_ricker.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, P]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class _Bound:
    """Keeps the converted arrays alive while the C struct points at them."""

    def __init__(self, g, amp=1.0):
        self.src_iz, self.src_ix = _i32(g.src_iz), _i32(g.src_ix)
        self.nt, self.rec_off = _i32(g.nt), _i32(g.rec_off)
        self.rec_iz, self.rec_ix = _i32(g.rec_iz), _i32(g.rec_ix)
        S = len(self.src_iz)
        assert len(self.src_ix) == S and len(self.nt) == S and len(self.rec_off) == S + 1
        assert float(g.freq) > 0.0, "the geometry must name the Ricker centre frequency"
        self.S = S
        self.nz, self.nx = int(g.nz), int(g.nx)
        self.st = _Geom(int(g.nz), int(g.nx), int(g.nb), float(g.dz), float(g.dx), float(g.dt), S,
                        _ptr(self.src_iz).value, _ptr(self.src_ix).value, _ptr(self.nt).value,
                        _ptr(self.rec_off).value, _ptr(self.rec_iz).value, _ptr(self.rec_ix).value,
                        float(g.freq), float(amp))

    @property
    def ref(self):
        return ctypes.byref(self.st)


def trace_count(g):
    nt = np.asarray(g.nt, dtype=np.int64)
    nrec = np.diff(np.asarray(g.rec_off, dtype=np.int64))
    return int((nt * nrec).sum())


def trace_offsets(g):
    nt = np.asarray(g.nt, dtype=np.int64)
    nrec = np.diff(np.asarray(g.rec_off, dtype=np.int64))
    return np.concatenate([[0], np.cumsum(nt * nrec)])


def num_threads():
    return lib().og_num_threads()


def ricker(f, dt, nt):
    """The oracle's source time function: w(n dt), n < nt, Ricker wavelet of
    centre frequency f delayed by 1.5/f (Sec. 4.1 reading)."""
    out = np.empty(int(nt))
    lib().og_ricker(float(f), float(dt), int(nt), _ptr(out))
    return out


# --------------------------------------------------------------------------
# Building blocks (Sec. 2.2 discretised; readings stated in oracle.c)
# --------------------------------------------------------------------------

def laplacian(u, dz, dx):
    """8th-order Laplacian of a 2D array, zero outside it."""
    u = _f64(u)
    out = np.empty_like(u)
    lib().og_laplacian(u.shape[0], u.shape[1], float(dz), float(dx), _ptr(u), _ptr(out))
    return out


def sponge(nz, nx, nb):
    """Cerjan damping factor G on the padded (nz+2nb) x (nx+2nb) grid."""
    G = np.empty((nz + 2 * nb, nx + 2 * nb))
    lib().og_sponge(nz, nx, nb, _ptr(G))
    return G


def extend(phys, nb):
    """Extension E: edge-replicate a physical field into the sponge."""
    phys = _f64(phys)
    nz, nx = phys.shape
    pad = np.empty((nz + 2 * nb, nx + 2 * nb))
    lib().og_extend(nz, nx, nb, _ptr(phys), _ptr(pad))
    return pad


def extend_adjoint(pad, nb):
    """E^T: fold sponge cells back onto the physical cells they replicate."""
    pad = _f64(pad)
    nz, nx = pad.shape[0] - 2 * nb, pad.shape[1] - 2 * nb
    phys = np.empty((nz, nx))
    lib().og_extend_adjoint(nz, nx, nb, _ptr(pad), _ptr(phys))
    return phys


def propagate(W, G, dz, dx, s, riz, rix):
    """Forward recurrence with a general source s[nt, NZ, NX] -> traces[nt, nrec]."""
    W, G, s = _f64(W), _f64(G), _f64(s)
    riz, rix = _i32(riz), _i32(rix)
    nt = s.shape[0]
    tr = np.empty((nt, len(riz)))
    lib().og_propagate(W.shape[0], W.shape[1], float(dz), float(dx), _ptr(W), _ptr(G), nt,
                       _ptr(s), len(riz), _ptr(riz), _ptr(rix), _ptr(tr))
    return tr


def propagate_adjoint(W, G, dz, dx, r, riz, rix):
    """Transpose of ``propagate``: traces r[nt, nrec] -> z[nt, NZ, NX]."""
    W, G, r = _f64(W), _f64(G), _f64(r)
    riz, rix = _i32(riz), _i32(rix)
    nt = r.shape[0]
    z = np.empty((nt,) + W.shape)
    lib().og_propagate_adjoint(W.shape[0], W.shape[1], float(dz), float(dx), _ptr(W), _ptr(G),
                               nt, _ptr(r), len(riz), _ptr(riz), _ptr(rix), _ptr(z))
    return z


# --------------------------------------------------------------------------
# Shot-level operators
# --------------------------------------------------------------------------

def forward(g, m, amp=1.0):
    """F: m (physical, s^2/m^2) -> traces  (eq. FWD sampled by R, eq. FWI);
    ``amp`` scales the source (linearity pins)."""
    b = _Bound(g, amp)
    m = _f64(m)
    assert m.shape == (b.nz, b.nx)
    out = np.empty(trace_count(g))
    lib().og_forward(b.ref, _ptr(m), _ptr(out))
    return out


def fwi_gradient(g, m, d_obs, want_resid=False):
    """(J, dJ/dm[, residual]) for J = 1/2||F(m) - d_obs||^2 (eqs. FWI, FWI_adj, adj_grad1)."""
    b = _Bound(g)
    m, d_obs = _f64(m), _f64(d_obs)
    assert m.shape == (b.nz, b.nx) and d_obs.size == trace_count(g)
    grad = np.empty((b.nz, b.nx))
    resid = np.empty(trace_count(g)) if want_resid else None
    J = lib().og_fwi_gradient(b.ref, _ptr(m), _ptr(d_obs), _ptr(grad), _ptr(resid))
    return (J, grad, resid) if want_resid else (J, grad)


def born_forward(g, m0, rho):
    """L: rho (dimensionless, m_r = rho*m0) -> scattered traces (eq. Born)."""
    b = _Bound(g)
    m0, rho = _f64(m0), _f64(rho)
    out = np.empty(trace_count(g))
    lib().og_born_forward(b.ref, _ptr(m0), _ptr(rho), _ptr(out))
    return out


def born_adjoint(g, m0, resid):
    """L^T: residual traces -> image on the physical grid (RTM when resid = d_r)."""
    b = _Bound(g)
    m0, resid = _f64(m0), _f64(resid)
    img = np.empty((b.nz, b.nx))
    lib().og_born_adjoint(b.ref, _ptr(m0), _ptr(resid), _ptr(img))
    return img


def lsrtm_gradient(g, m0, rho, d_obs):
    """(J, grad) for J(rho) = 1/2||L rho - d_obs||^2 (eq. LSRTM): grad = L^T(L rho - d_obs)."""
    r = born_forward(g, m0, rho) - _f64(d_obs)
    return 0.5 * float(r @ r), born_adjoint(g, m0, r)
