"""Thin ctypes binding of libaafwi.so (include/aafwi.h).

Argument marshalling only: tensors are passed as raw device pointers with the
current torch CUDA stream; every computation runs in the library's CUDA
kernels.  There is no CPU fallback: if the library cannot be loaded the
import of the symbols raises.
"""
import ctypes
import hashlib
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libaafwi.so")

AAFWI_OK = 0
ERR_NAMES = {1: "ARG", 2: "CFL", 3: "OOB", 4: "NAN", 5: "TIMEOUT", 6: "CUDA", 7: "NOMEM", 8: "STATE"}
MODE_FWI = 0
MODE_LSRTM = 1
REUSE_FORWARD = 1

# every entry point declared in include/aafwi.h
EXPORTS = ("aafwi_plan_create", "aafwi_plan_destroy", "aafwi_plan_get_info", "aafwi_last_error",
           "aafwi_plan_set_stall",
           "aafwi_model_forward", "aafwi_born_forward", "aafwi_misfit", "aafwi_adjoint_gradient",
           "aafwi_adjoint_gradient_host",
           "aafwi_born_adjoint", "aafwi_fwi_adjoint", "aafwi_read_misfit", "aafwi_aa_create", "aafwi_aa_destroy",
           "aafwi_aa_set_eta", "aafwi_aa_set_beta", "aafwi_aa_set_weights", "aafwi_aa_step", "aafwi_aa_combine", "aafwi_absmax",
           "aafwi_launch_count", "aafwi_misfit_noalloc", "aafwi_unet_create", "aafwi_unet_destroy",
           "aafwi_unet_param_count", "aafwi_unet_set_params", "aafwi_unet_get_params", "aafwi_unet_forward",
           "aafwi_unet_loss_grad", "aafwi_unet_train_step", "aafwi_learned_features", "aafwi_learned_apply",
           "aafwi_autotune", "aafwi_dot", "aafwi_axpby", "aafwi_aa_set_norm", "aafwi_aa_get_lp_info",
           "aafwi_lp_min", "aafwi_axpby_clip", "aafwi_unet_conv3x3")

NORM_L2, NORM_L1, NORM_LINF = 0, 1, 2
CONV3_FWD, CONV3_DGRAD, CONV3_WGRAD = 0, 1, 2


class AafwiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("aafwi error %s (%d): %s" % (ERR_NAMES.get(code, "?"), code, msg))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("nb", ctypes.c_int),
                ("dx", ctypes.c_double), ("dz", ctypes.c_double), ("dt", ctypes.c_double),
                ("c_max", ctypes.c_double)]


class Shots(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("src_iz", ctypes.c_void_p), ("src_ix", ctypes.c_void_p),
                ("nt", ctypes.c_void_p), ("rec_off", ctypes.c_void_p),
                ("rec_iz", ctypes.c_void_p), ("rec_ix", ctypes.c_void_p)]


ENGINE_AUTO, ENGINE_PER_STEP, ENGINE_PERSISTENT, ENGINE_HYBRID = 0, 1, 2, 3


class PlanOpts(ctypes.Structure):
    _fields_ = [("max_workspace_bytes", ctypes.c_size_t), ("checkpoint_every", ctypes.c_int),
                ("tile_z", ctypes.c_int), ("tile_x", ctypes.c_int), ("engine", ctypes.c_int),
                ("no_graphs", ctypes.c_int), ("shots_per_batch", ctypes.c_int), ("no_pdl", ctypes.c_int),
                ("steps_per_launch", ctypes.c_int), ("lanes", ctypes.c_int), ("l2_batches", ctypes.c_int)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("engine", ctypes.c_int), ("tile_z", ctypes.c_int), ("lanes", ctypes.c_int),
                ("ms", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("NZ", ctypes.c_int), ("NX", ctypes.c_int), ("pitch", ctypes.c_int),
                ("S", ctypes.c_int), ("nt_max", ctypes.c_int), ("trace_count", ctypes.c_longlong),
                ("checkpoint_every", ctypes.c_int), ("n_checkpoints", ctypes.c_int),
                ("workspace_bytes", ctypes.c_size_t), ("tile_z", ctypes.c_int),
                ("tile_x", ctypes.c_int), ("n_tiles", ctypes.c_int), ("engine", ctypes.c_int),
                ("persist_ctas", ctypes.c_int), ("shots_per_batch", ctypes.c_int), ("n_batches", ctypes.c_int),
                ("steps_per_launch", ctypes.c_int), ("lanes", ctypes.c_int)]


_lib = None


def load(path=LIB_PATH):
    """Load libaafwi.so (raises OSError if it is missing: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libaafwi.so not built (%s); run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    P, I, D, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "aafwi_plan_create": ([P, P, P, P, P], I),
        "aafwi_plan_destroy": ([P], None),
        "aafwi_plan_get_info": ([P, P], I),
        "aafwi_plan_set_stall": ([P, I], I),
        "aafwi_last_error": ([P], ctypes.c_char_p),
        "aafwi_model_forward": ([P, P, P, P], I),
        "aafwi_born_forward": ([P, P, P, P, P], I),
        "aafwi_misfit": ([P, P, P, P, P, P], I),
        "aafwi_adjoint_gradient": ([P, I, P, P, P, P, P, I, P], I),
        "aafwi_adjoint_gradient_host": ([P, I, P, P, P, P, P, P], I),
        "aafwi_born_adjoint": ([P, P, P, P, P], I),
        "aafwi_fwi_adjoint": ([P, P, P, P, I, P], I),
        "aafwi_read_misfit": ([P, P, P], I),
        "aafwi_aa_create": ([Z, I, D, P], I),
        "aafwi_aa_destroy": ([P], None),
        "aafwi_aa_set_eta": ([P, D], I),
        "aafwi_aa_set_beta": ([P, D], I),
        "aafwi_aa_set_weights": ([P, P, P], I),
        "aafwi_aa_step": ([P, P, P, P, P, P, P, P], I),
        "aafwi_aa_combine": ([P, D, P, P, P, ctypes.c_float, ctypes.c_float, P, P], I),
        "aafwi_absmax": ([P, Z, P, P], I),
        "aafwi_launch_count": ([], ctypes.c_ulonglong),
        "aafwi_misfit_noalloc": ([P, P, ctypes.c_longlong, P, P, P, P], I),
        "aafwi_unet_create": ([I, I, I, I, P], I),
        "aafwi_unet_destroy": ([P], None),
        "aafwi_unet_param_count": ([P], ctypes.c_longlong),
        "aafwi_unet_set_params": ([P, P, ctypes.c_longlong], I),
        "aafwi_unet_get_params": ([P, P, ctypes.c_longlong], I),
        "aafwi_unet_forward": ([P, P, I, P, P], I),
        "aafwi_unet_loss_grad": ([P, P, P, I, P, P, P], I),
        "aafwi_unet_train_step": ([P, P, P, I, ctypes.c_float, P, P], I),
        "aafwi_unet_conv3x3": ([I, P, P, I, I, I, I, I, I, P, ctypes.c_longlong, ctypes.POINTER(I), P], I),
        "aafwi_learned_features": ([P, P, I, I, I, I, P, P, P], I),
        "aafwi_learned_apply": ([P, P, I, I, I, P, ctypes.c_float, ctypes.c_float, P, P], I),
        "aafwi_autotune": ([P, P, P, P, I, I, P, P, I, P, P], I),
        "aafwi_dot": ([P, P, Z, P, P], I),
        "aafwi_axpby": ([D, P, D, P, Z, P], I),
        "aafwi_aa_set_norm": ([P, I], I),
        "aafwi_aa_get_lp_info": ([P, P], I),
        "aafwi_lp_min": ([I, I, P, P, P, P, P], I),
        "aafwi_axpby_clip": ([D, P, D, P, Z, ctypes.c_float, ctypes.c_float, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(rc, plan=None):
    if rc != AAFWI_OK:
        msg = load().aafwi_last_error(plan)
        raise AafwiError(rc, msg.decode() if msg else "")


def _ptr(t):
    """Device pointer of a contiguous CUDA float32 tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _f32(t):
    import torch
    if t.dtype != torch.float32:
        raise TypeError("expected float32, got %s" % t.dtype)
    return _ptr(t)


def _host_f32(t):
    """Host pointer of a contiguous CPU float32 tensor (None -> NULL)."""
    import torch
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous() or t.dtype != torch.float32:
        raise ValueError("expected a contiguous CPU float32 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _geom_structs(geom, c_max):
    """(Grid, Shots, arrays kept alive) of a geometry; the last kept array is
    the FP64 wavelet."""
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    keep = [i32(geom.src_iz), i32(geom.src_ix), i32(geom.nt), i32(geom.rec_off),
            i32(geom.rec_iz), i32(geom.rec_ix), np.ascontiguousarray(geom.wavelet, dtype=np.float64)]
    g = Grid(int(geom.nx), int(geom.nz), int(geom.nb), float(geom.dx), float(geom.dz),
             float(geom.dt), float(c_max))
    s = Shots(len(keep[0]), *[_np_ptr(a) for a in keep[:6]])
    return g, s, keep


# ---- autotuner ---------------------------------------------------------------

def tune_key(geom, c_max, device_name, sm_count, engine=ENGINE_AUTO, max_workspace_bytes=0):
    """Cache key of a tuning: the device and everything the plan's launch
    configuration depends on (grid, shots, receivers, record lengths)."""
    h = hashlib.sha1()
    for a in (geom.src_iz, geom.src_ix, geom.nt, geom.rec_off, geom.rec_iz, geom.rec_ix):
        h.update(np.ascontiguousarray(a, dtype=np.int32).tobytes())
    return "%s|sm%d|%dx%d|nb%d|S%d|nt%d|e%d|ws%d|%s" % (
        device_name, int(sm_count), int(geom.nx), int(geom.nz), int(geom.nb), len(geom.src_iz),
        int(np.max(geom.nt)), int(engine), int(max_workspace_bytes), h.hexdigest()[:16])


def default_tune_cache():
    return os.environ.get("AAFWI_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "aafwi", "tune.json"))


def cache_lookup(path, key):
    try:
        with open(path) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def cache_store(path, key, value):
    """Add one entry (read-modify-write, replaced atomically)."""
    data = {}
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[key] = value
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = "%s.%d.tmp" % (path, os.getpid())
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def run_autotune(geom, c_max, m, steps=64, reps=3, engine=ENGINE_AUTO, max_workspace_bytes=0):
    """aafwi_autotune: {"engine", "tile_z", "lanes", "table": [(engine, tile_z, lanes, ms), ...]}."""
    L = load()
    g, s, keep = _geom_structs(geom, c_max)
    base = PlanOpts(int(max_workspace_bytes), 0, 0, 0, int(engine), 0, 0)
    best = PlanOpts()
    table = (TuneEntry * 16)()
    n = ctypes.c_int()
    _check(L.aafwi_autotune(ctypes.byref(g), ctypes.byref(s), _np_ptr(keep[6]), _f32(m), int(steps),
                            int(reps), ctypes.byref(base), table, 16, ctypes.byref(n), ctypes.byref(best)))
    return {"engine": int(best.engine), "tile_z": int(best.tile_z), "lanes": int(best.lanes), "steps": int(steps),
            "table": [(int(table[i].engine), int(table[i].tile_z), int(table[i].lanes), float(table[i].ms))
                      for i in range(n.value)]}


def autotune(geom, c_max, m, steps=64, reps=3, engine=ENGINE_AUTO, max_workspace_bytes=0, cache_path=None,
             tuner=None, device=None):
    """Launch configuration for plans of this geometry on this device: from the
    cache when present, else timed by the library (and stored)."""
    if device is None:
        import torch
        prop = torch.cuda.get_device_properties(m.device)
        device = (prop.name, prop.multi_processor_count)
    path = cache_path or default_tune_cache()
    key = tune_key(geom, c_max, device[0], device[1], engine, max_workspace_bytes)
    hit = cache_lookup(path, key)
    if hit is not None:
        return dict(hit, cached=True)
    tuner = tuner or run_autotune
    res = json.loads(json.dumps(tuner(geom, c_max, m, steps=steps, reps=reps, engine=engine,
                                      max_workspace_bytes=max_workspace_bytes)))   # as stored
    cache_store(path, key, res)
    return dict(res, cached=False)


class Plan:
    """Owns an aafwi_plan: geometry, workspace and the wave-equation operators."""

    def __init__(self, geom, c_max, max_workspace_bytes=0, checkpoint_every=0, engine=ENGINE_AUTO,
                 graphs=True, tile_z=0, tune_model=None, tune_cache=None, shots_per_batch=0, pdl=True,
                 steps_per_launch=0, lanes=0, l2_batches=0):
        """tune_model: a device model m [nz][nx]; when given, the engine and
        tile height (and the shot lanes, unless given) come from autotune() (cached in tune_cache, default
        $AAFWI_TUNE_CACHE or ~/.cache/aafwi/tune.json)."""
        L = load()
        self.geom = geom
        if tune_model is not None:
            t = autotune(geom, c_max, tune_model, engine=engine, max_workspace_bytes=max_workspace_bytes,
                         cache_path=tune_cache)
            engine, tile_z = t["engine"], t["tile_z"]
            lanes = lanes or t.get("lanes", 0)
            self.tuning = t
        g, s, self._keep = _geom_structs(geom, c_max)
        o = PlanOpts(int(max_workspace_bytes), int(checkpoint_every), int(tile_z), 0, int(engine),
                     0 if graphs else 1, int(shots_per_batch), 0 if pdl else 1, int(steps_per_launch),
                     int(lanes), int(l2_batches))
        h = ctypes.c_void_p()
        _check(L.aafwi_plan_create(ctypes.byref(g), ctypes.byref(s), _np_ptr(self._keep[6]),
                                   ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        info = PlanInfo()
        _check(L.aafwi_plan_get_info(h, ctypes.byref(info)), h)
        self.info = info
        self.trace_count = int(info.trace_count)
        self.keeps_forward = info.n_batches == 1   # the stored forward can be reused (REUSE_FORWARD)

    def close(self):
        if getattr(self, "h", None):
            load().aafwi_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stall(self, step):
        """Failure-detection test hook (see aafwi_plan_set_stall)."""
        _check(load().aafwi_plan_set_stall(self.h, int(step)), self.h)

    # --- operators ---------------------------------------------------------
    def model_forward(self, m, d_out=None, stream=None):
        _check(load().aafwi_model_forward(self.h, _f32(m), _f32(d_out) if d_out is not None else None,
                                          _stream(stream)), self.h)
        return d_out

    def born_forward(self, m0, rho, d_out, stream=None):
        _check(load().aafwi_born_forward(self.h, _f32(m0), _f32(rho), _f32(d_out), _stream(stream)), self.h)
        return d_out

    def misfit(self, d_syn, d_obs, resid=None, sync=True, stream=None):
        J = ctypes.c_double()
        _check(load().aafwi_misfit(self.h, _f32(d_syn), _f32(d_obs),
                                   _f32(resid) if resid is not None else None,
                                   ctypes.byref(J) if sync else None, _stream(stream)), self.h)
        return J.value if sync else None

    def adjoint_gradient(self, mode, m, rho, d_obs, grad, sync=True, reuse_forward=False, stream=None):
        J = ctypes.c_double()
        _check(load().aafwi_adjoint_gradient(self.h, int(mode), _f32(m),
                                             _f32(rho) if rho is not None else None, _f32(d_obs),
                                             _f32(grad), ctypes.byref(J) if sync else None,
                                             REUSE_FORWARD if reuse_forward else 0, _stream(stream)),
               self.h)
        return J.value if sync else None

    def adjoint_gradient_host(self, mode, m, rho, d_obs, grad, stream=None):
        """adjoint_gradient with host (CPU) tensors, copies included; returns J."""
        J = ctypes.c_double()
        _check(load().aafwi_adjoint_gradient_host(self.h, int(mode), _host_f32(m), _host_f32(rho),
                                                  _host_f32(d_obs), _host_f32(grad), ctypes.byref(J),
                                                  _stream(stream)), self.h)
        return J.value

    def fwi_adjoint(self, m, adj_src, grad, reuse_forward=False, stream=None):
        _check(load().aafwi_fwi_adjoint(self.h, _f32(m), _f32(adj_src), _f32(grad),
                                        REUSE_FORWARD if reuse_forward else 0, _stream(stream)), self.h)
        return grad

    def born_adjoint(self, m0, resid, img, stream=None):
        _check(load().aafwi_born_adjoint(self.h, _f32(m0), _f32(resid), _f32(img), _stream(stream)), self.h)
        return img

    def read_misfit(self, stream=None):
        J = ctypes.c_double()
        _check(load().aafwi_read_misfit(self.h, ctypes.byref(J), _stream(stream)), self.h)
        return J.value


def dot(x, y, stream=None):
    """<x, y> (FP64 accumulation) of two contiguous device float32 tensors."""
    out = ctypes.c_double()
    _check(load().aafwi_dot(_f32(x), _f32(y), x.numel(), ctypes.byref(out), _stream(stream)))
    return out.value


def axpby(a, x, b, y, stream=None):
    """y <- a x + b y in place (device float32)."""
    _check(load().aafwi_axpby(float(a), _f32(x), float(b), _f32(y), y.numel(), _stream(stream)))
    return y


def axpby_clip(a, x, b, y, lo, hi, stream=None):
    """y <- clip(a x + b y, lo, hi) in place (device float32; no clip when lo >= hi)."""
    _check(load().aafwi_axpby_clip(float(a), _f32(x), float(b), _f32(y), y.numel(), float(lo), float(hi),
                                   _stream(stream)))
    return y


class AA:
    """Owns an aafwi_aa: the AA(M) history ring and its FP64 Gram matrix."""

    def __init__(self, n, M, eta):
        h = ctypes.c_void_p()
        _check(load().aafwi_aa_create(int(n), int(M), float(eta), ctypes.byref(h)))
        self.h, self.n, self.M = h, int(n), int(M)

    def close(self):
        if getattr(self, "h", None):
            load().aafwi_aa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_eta(self, eta):
        _check(load().aafwi_aa_set_eta(self.h, float(eta)))

    def set_weights(self, w, stream=None):
        """Weighted l2 norm of the AA least squares (None: plain l2); before the first step."""
        _check(load().aafwi_aa_set_weights(self.h, _f32(w) if w is not None else None, _stream(stream)))

    def set_beta(self, beta):
        """Damping of the AA point (Alg. 1 eq. AAupdate0); 1 = Alg. 2."""
        _check(load().aafwi_aa_set_beta(self.h, float(beta)))

    def set_norm(self, norm):
        """Norm of the optimisation step (Sec. 2.1): NORM_L2, NORM_L1 or NORM_LINF."""
        _check(load().aafwi_aa_set_norm(self.h, int(norm)))

    def lp_info(self):
        """Statistics of the last l1 / l-infinity step (aafwi_aa_lp_info as a dict)."""
        info = AALpInfo()
        _check(load().aafwi_aa_get_lp_info(self.h, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in AALpInfo._fields_}

    def step(self, p_k, grad_k, p_tilde, p_bar, want_gamma=False, stream=None):
        gam = (ctypes.c_double * max(self.M, 1))()
        Mk = ctypes.c_int()
        _check(load().aafwi_aa_step(self.h, _f32(p_k), _f32(grad_k), _f32(p_tilde), _f32(p_bar),
                                    gam if want_gamma else None,
                                    ctypes.byref(Mk) if want_gamma else None, _stream(stream)))
        if want_gamma:
            return np.array(gam[:Mk.value]), Mk.value
        return None

    def combine(self, lam, p_tilde, p_bar, p_next, lo=0.0, hi=0.0, want_dot=False, stream=None):
        dot = ctypes.c_double()
        _check(load().aafwi_aa_combine(self.h, float(lam), _f32(p_tilde), _f32(p_bar), _f32(p_next),
                                       float(lo), float(hi), ctypes.byref(dot) if want_dot else None,
                                       _stream(stream)))
        return dot.value if want_dot else None


class AALpInfo(ctypes.Structure):
    _fields_ = [("objective", ctypes.c_double), ("lower_bound", ctypes.c_double),
                ("rounds", ctypes.c_int), ("rows", ctypes.c_int)]


def unet_conv3x3(op, a, b, B, H, W, Cin, Cout, splits=0, max_splits=None, stream=None):
    """aafwi_unet_conv3x3: one 3x3 convolution GEMM of the U-Net on BF16 device
    tensors (NHWC activations; weights [Cout][3][3][Cin], or [Cin][3][3][Cout]
    for CONV3_DGRAD).  Returns the FP32 split slices [s][...] (their sum is the
    result) and s."""
    import torch
    for t in (a, b):
        if t.dtype != torch.bfloat16 or not t.is_cuda or not t.is_contiguous():
            raise TypeError("expected contiguous CUDA bfloat16 tensors")
    P = B * H * W
    MN = 9 * Cin * Cout if op == CONV3_WGRAD else P * (Cout if op == CONV3_FWD else Cin)
    if max_splits is None:
        max_splits = 256 if op == CONV3_WGRAD else 8
    cap = max(1, max_splits if splits <= 0 else min(splits, max_splits))
    out = torch.empty(cap * MN, device=a.device, dtype=torch.float32)
    s = ctypes.c_int(0)
    _check(load().aafwi_unet_conv3x3(int(op), ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                     int(B), int(H), int(W), int(Cin), int(Cout), int(splits),
                                     ctypes.c_void_p(out.data_ptr()), cap * MN, ctypes.byref(s), _stream(stream)))
    return out[:s.value * MN].view(s.value, -1), s.value


def lp_min(A, b, c):
    """aafwi_lp_min (host only): argmin c^T x s.t. A x <= b; returns (x, c^T x)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    m, nv = A.shape
    x = np.empty(nv)
    obj = ctypes.c_double()
    _check(load().aafwi_lp_min(nv, m, A.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p),
                               c.ctypes.data_as(ctypes.c_void_p), x.ctypes.data_as(ctypes.c_void_p),
                               ctypes.byref(obj)))
    return x, obj.value


MISFIT_NOALLOC_MAX_SAMPLES = 1 << 32


def misfit_noalloc(d_syn, d_obs, resid=None, J_dev=None, sync=True, n=None, stream=None):
    """aafwi_misfit_noalloc: the misfit with the library's static scratch (no
    device allocation; for callers that cannot allocate).  Returns J (sync)."""
    J = ctypes.c_double()
    n = d_syn.numel() if n is None else int(n)
    _check(load().aafwi_misfit_noalloc(_f32(d_syn), _f32(d_obs), n,
                                       _f32(resid) if resid is not None else None,
                                       _ptr(J_dev) if J_dev is not None else None,
                                       ctypes.byref(J) if sync else None, _stream(stream)))
    return J.value if sync else None


class UNet:
    """Owns an aafwi_unet (the learned preconditioner's network)."""

    def __init__(self, Bmax, H, W, C=32):
        h = ctypes.c_void_p()
        _check(load().aafwi_unet_create(int(Bmax), int(H), int(W), int(C), ctypes.byref(h)))
        self.h, self.Bmax, self.H, self.W, self.C = h, int(Bmax), int(H), int(W), int(C)
        self.nparam = int(load().aafwi_unet_param_count(h))

    def close(self):
        if getattr(self, "h", None):
            load().aafwi_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == self.nparam
        _check(load().aafwi_unet_set_params(self.h, a.ctypes.data_as(ctypes.c_void_p), a.size))

    def get_params(self):
        a = np.empty(self.nparam, dtype=np.float32)
        _check(load().aafwi_unet_get_params(self.h, a.ctypes.data_as(ctypes.c_void_p), a.size))
        return a

    def forward(self, x, y=None, stream=None):
        import torch
        B = x.shape[0]
        if y is None:
            y = torch.empty((B, self.H, self.W), dtype=torch.float32, device=x.device)
        _check(load().aafwi_unet_forward(self.h, _f32(x), B, _f32(y), _stream(stream)))
        return y

    def loss_grad(self, x, target, grad=None, stream=None):
        J = ctypes.c_double()
        _check(load().aafwi_unet_loss_grad(self.h, _f32(x), _f32(target), x.shape[0],
                                           _f32(grad) if grad is not None else None, ctypes.byref(J),
                                           _stream(stream)))
        return J.value

    def train_step(self, x, target, lr, stream=None):
        J = ctypes.c_double()
        _check(load().aafwi_unet_train_step(self.h, _f32(x), _f32(target), x.shape[0], float(lr),
                                            ctypes.byref(J), _stream(stream)))
        return J.value


def learned_features(grad, m, H, W, x, stats, stream=None):
    """aafwi_learned_features: network input x[2][H][W] and stats (device double[3])."""
    nz, nx = m.shape
    _check(load().aafwi_learned_features(_f32(grad), _f32(m), nz, nx, int(H), int(W), _f32(x), _ptr(stats),
                                         _stream(stream)))


def learned_apply(m, delta, stats, out, lo=0.0, hi=0.0, stream=None):
    """aafwi_learned_apply: out = clip(m + std_m * delta)."""
    nz, nx = m.shape
    _check(load().aafwi_learned_apply(_f32(m), _f32(delta), nz, nx, int(delta.shape[-1]), _ptr(stats),
                                      float(lo), float(hi), _f32(out), _stream(stream)))


def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(load().aafwi_launch_count())


def absmax(x, stream=None):
    out = ctypes.c_double()
    _check(load().aafwi_absmax(_f32(x), x.numel(), ctypes.byref(out), _stream(stream)))
    return out.value
