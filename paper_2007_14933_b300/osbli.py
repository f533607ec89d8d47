"""Thin ctypes binding of include/osbli.h (argument marshalling only).

Every numerical step runs in libosbli.so; this module only converts arguments.  Functions keep the
C names (``osbli_create`` ...); ``Solver`` wraps a handle for convenience.  Arrays may be numpy
arrays (host memory) or torch tensors (device or pinned host memory); layouts are those of the
header: state [5][nz][ny][nx] FP64 contiguous.

Loading fails loudly (OSError) when the library has not been built: there is no fallback path.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libosbli.so")

OSBLI_OK, OSBLI_EINVAL, OSBLI_ENOMEM, OSBLI_ECUDA, OSBLI_ENONFINITE, OSBLI_ETIMEOUT, OSBLI_ESTATE = \
    0, -1, -2, -3, -4, -5, -6
OSBLI_CENTRAL4, OSBLI_WENO5JS, OSBLI_TENO5, OSBLI_WENO5Z, OSBLI_TENO6 = 0, 1, 2, 3, 4
OSBLI_PERIODIC, OSBLI_ZEROGRAD, OSBLI_WALL, OSBLI_DIRICHLET, OSBLI_INFLOW, OSBLI_ADIABATIC = 0, 1, 2, 3, 4, 5
OSBLI_FP64, OSBLI_MIXED = 0, 1
OSBLI_RK3, OSBLI_RK4, OSBLI_SSPRK3 = 0, 1, 2

EXPORTED = ["osbli_create", "osbli_destroy", "osbli_set_boundary_data", "osbli_set_state",
            "osbli_get_state", "osbli_rk_step", "osbli_residual", "osbli_diagnostics",
            "osbli_launches_per_step", "osbli_last_error", "osbli_profile_residual",
            "osbli_profile_name", "osbli_fp64_peak", "osbli_residual_noalloc",
            "osbli_fp32_peak", "osbli_sensor_set_weights", "osbli_sensor_set_gate", "osbli_sensor_labels",
            "osbli_sensor_features", "osbli_sensor_probs", "osbli_mlp_grad", "osbli_mlp_train",
            "osbli_mlp_forward", "osbli_ensemble_create", "osbli_ensemble_destroy",
            "osbli_ensemble_set_state", "osbli_ensemble_get_state", "osbli_ensemble_member",
            "osbli_ensemble_step", "osbli_ensemble_set_chunk", "osbli_ensemble_autotune",
            "osbli_ensemble_launches_per_step", "osbli_ensemble_points", "osbli_ensemble_last_error",
            "osbli_domain_plan", "osbli_domain_create", "osbli_domain_destroy", "osbli_domain_set_state",
            "osbli_domain_get_state", "osbli_domain_set_boundary_data", "osbli_domain_step",
            "osbli_domain_residual", "osbli_domain_slabs", "osbli_domain_member",
            "osbli_domain_launches_per_step", "osbli_domain_last_error", "osbli_ensemble_set_persistent",
            "osbli_ensemble_persistent_grid"]
DOMAIN_MAX_SLABS = 64
SENSOR_NPARAM = 5441
SENSOR_NFEAT = 144


class osbli_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("gamma", ctypes.c_double), ("Re", ctypes.c_double), ("Pr", ctypes.c_double),
        ("Ma", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("teno_ct", ctypes.c_double),
        ("bc", (ctypes.c_int * 2) * 3),
        ("T_wall", ctypes.c_double),
        ("sutherland_ratio", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("sensor", ctypes.c_int),
        ("h", ctypes.c_double * 3),
        ("L", ctypes.c_double * 3),
        ("rk", ctypes.c_int),
        ("force", ctypes.c_double * 3),
    ]


class OsbliError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("osbli error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load():
    """Load libosbli.so (raises OSError when it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libosbli.so not built (run paper_2007_14933_b300/build.py): %s" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.osbli_create.argtypes = [ctypes.POINTER(osbli_params), vp, vp, ctypes.POINTER(vp)]
        L.osbli_destroy.argtypes = [vp]
        L.osbli_destroy.restype = None
        L.osbli_set_boundary_data.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
        L.osbli_set_state.argtypes = [vp, vp]
        L.osbli_get_state.argtypes = [vp, vp]
        L.osbli_rk_step.argtypes = [vp, ctypes.c_int]
        L.osbli_residual.argtypes = [vp, vp]
        L.osbli_diagnostics.argtypes = [vp, vp]
        L.osbli_launches_per_step.argtypes = [vp]
        L.osbli_profile_residual.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
        L.osbli_profile_name.argtypes = [vp, ctypes.c_int]
        L.osbli_profile_name.restype = ctypes.c_char_p
        L.osbli_residual_noalloc.argtypes = [ctypes.POINTER(osbli_params), vp, vp, vp]
        L.osbli_residual_noalloc.restype = ctypes.c_int
        L.osbli_sensor_set_weights.argtypes = [vp, vp, ctypes.c_float]
        L.osbli_sensor_set_gate.argtypes = [vp, vp]
        L.osbli_sensor_set_gate.restype = ctypes.c_int
        L.osbli_sensor_labels.argtypes = [vp, vp]
        L.osbli_sensor_features.argtypes = [vp, vp]
        L.osbli_sensor_probs.argtypes = [vp, vp]
        L.osbli_mlp_grad.argtypes = [vp, vp, ctypes.c_longlong, ctypes.c_float, vp, vp,
                                     ctypes.POINTER(ctypes.c_double)]
        L.osbli_mlp_train.argtypes = [vp, vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_float, ctypes.c_float, ctypes.c_uint, vp, vp]
        L.osbli_mlp_forward.argtypes = [vp, ctypes.c_longlong, vp, vp]
        L.osbli_mlp_forward.restype = ctypes.c_int
        for name in ("osbli_sensor_set_weights", "osbli_sensor_labels", "osbli_sensor_features",
                     "osbli_sensor_probs", "osbli_mlp_grad", "osbli_mlp_train"):
            getattr(L, name).restype = ctypes.c_int
        L.osbli_fp64_peak.argtypes = [ctypes.POINTER(ctypes.c_double)]
        L.osbli_fp64_peak.restype = ctypes.c_int
        L.osbli_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double)]
        L.osbli_fp32_peak.restype = ctypes.c_int
        L.osbli_last_error.argtypes = [vp]
        L.osbli_last_error.restype = ctypes.c_char_p
        L.osbli_ensemble_create.argtypes = [ctypes.c_int, ctypes.POINTER(osbli_params), vp, ctypes.POINTER(vp)]
        L.osbli_ensemble_destroy.argtypes = [vp]
        L.osbli_ensemble_destroy.restype = None
        L.osbli_ensemble_set_state.argtypes = [vp, ctypes.c_int, vp]
        L.osbli_ensemble_get_state.argtypes = [vp, ctypes.c_int, vp]
        L.osbli_ensemble_member.argtypes = [vp, ctypes.c_int]
        L.osbli_ensemble_member.restype = vp
        L.osbli_ensemble_step.argtypes = [vp, ctypes.c_int]
        L.osbli_ensemble_set_chunk.argtypes = [vp, ctypes.c_int]
        L.osbli_ensemble_autotune.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_double)]
        L.osbli_ensemble_launches_per_step.argtypes = [vp]
        L.osbli_ensemble_points.argtypes = [vp]
        L.osbli_ensemble_points.restype = ctypes.c_longlong
        L.osbli_ensemble_set_persistent.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
        L.osbli_ensemble_set_persistent.restype = ctypes.c_int
        L.osbli_ensemble_persistent_grid.argtypes = [vp]
        L.osbli_ensemble_persistent_grid.restype = ctypes.c_int
        L.osbli_ensemble_last_error.argtypes = [vp]
        L.osbli_ensemble_last_error.restype = ctypes.c_char_p
        for name in ("osbli_ensemble_create", "osbli_ensemble_set_state", "osbli_ensemble_get_state",
                     "osbli_ensemble_step", "osbli_ensemble_set_chunk", "osbli_ensemble_autotune",
                     "osbli_ensemble_launches_per_step"):
            getattr(L, name).restype = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int)
        L.osbli_domain_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip, ip, ip]
        L.osbli_domain_create.argtypes = [ctypes.POINTER(osbli_params), ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.osbli_domain_destroy.argtypes = [vp]
        L.osbli_domain_destroy.restype = None
        L.osbli_domain_set_state.argtypes = [vp, vp]
        L.osbli_domain_get_state.argtypes = [vp, vp]
        L.osbli_domain_set_boundary_data.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
        L.osbli_domain_step.argtypes = [vp, ctypes.c_int]
        L.osbli_domain_residual.argtypes = [vp, vp]
        L.osbli_domain_slabs.argtypes = [vp]
        L.osbli_domain_member.argtypes = [vp, ctypes.c_int]
        L.osbli_domain_member.restype = vp
        L.osbli_domain_launches_per_step.argtypes = [vp, ip]
        L.osbli_domain_last_error.argtypes = [vp]
        L.osbli_domain_last_error.restype = ctypes.c_char_p
        for name in ("osbli_domain_plan", "osbli_domain_create", "osbli_domain_set_state",
                     "osbli_domain_get_state", "osbli_domain_set_boundary_data", "osbli_domain_step",
                     "osbli_domain_residual", "osbli_domain_slabs", "osbli_domain_launches_per_step"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("osbli_create", "osbli_set_boundary_data", "osbli_set_state", "osbli_get_state",
                     "osbli_rk_step", "osbli_residual", "osbli_diagnostics",
                     "osbli_launches_per_step", "osbli_profile_residual"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    """Address of a numpy array or torch tensor (contiguous FP64 expected)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data)


def _check(h, rc):
    if rc != OSBLI_OK:
        msg = load().osbli_last_error(h)
        raise OsbliError(rc, msg.decode() if msg else "")
    return rc


def make_params(cfg, precision=OSBLI_FP64):
    p = osbli_params()
    p.nx, p.ny, p.nz = (int(x) for x in cfg["n"])
    p.gamma = cfg.get("gamma", 1.4)
    p.Re = cfg.get("Re", 0.0)
    p.Pr = cfg.get("Pr", 0.72)
    p.Ma = cfg.get("Ma", 1.0)
    p.dt = cfg.get("dt", 0.0)
    p.scheme = int(cfg.get("scheme", OSBLI_TENO5))
    p.teno_ct = cfg.get("teno_ct", 1e-5)
    for d in range(3):
        for s in range(2):
            p.bc[d][s] = int(cfg["bc"][d][s])
        p.h[d] = float(cfg.get("h", (1.0, 1.0, 1.0))[d])
        p.L[d] = float(cfg.get("L", (0.0, 0.0, 0.0))[d])
    p.T_wall = cfg.get("T_wall", 1.0)
    p.sutherland_ratio = cfg.get("suth", 0.0)
    p.precision = int(precision)
    p.sensor = int(cfg.get("sensor", 0))
    p.rk = int(cfg.get("rk", 0))
    for q, f in enumerate(cfg.get("force", (0.0, 0.0, 0.0))):
        p.force[q] = float(f)
    return p


# ---- the C names ------------------------------------------------------------------------------
def osbli_create(params, coords=None, cuda_stream=None):
    h = ctypes.c_void_p()
    c = None if coords is None else np.ascontiguousarray(coords, dtype=np.float64)
    _check(None, load().osbli_create(ctypes.byref(params), _ptr(c), ctypes.c_void_p(cuda_stream or 0),
                                     ctypes.byref(h)))
    return h


def osbli_destroy(h):
    load().osbli_destroy(h)


def osbli_set_boundary_data(h, d, s, prims):
    return _check(h, load().osbli_set_boundary_data(h, int(d), int(s), _ptr(prims)))


def osbli_set_state(h, U):
    return _check(h, load().osbli_set_state(h, _ptr(U)))


def osbli_get_state(h, U):
    return _check(h, load().osbli_get_state(h, _ptr(U)))


def osbli_rk_step(h, nsteps):
    return _check(h, load().osbli_rk_step(h, int(nsteps)))


def osbli_residual(h, R):
    return _check(h, load().osbli_residual(h, _ptr(R)))


def osbli_diagnostics(h, out):
    return _check(h, load().osbli_diagnostics(h, _ptr(out)))


def osbli_launches_per_step(h):
    return load().osbli_launches_per_step(h)


def osbli_profile_residual(h, reps, max_launches=32):
    """Mean per-launch milliseconds of one residual evaluation: [(name, ms), ...]."""
    ms = np.zeros(max_launches)
    n = load().osbli_profile_residual(h, int(reps), _ptr(ms), max_launches)
    if n < 0:
        _check(h, n)
    return [(load().osbli_profile_name(h, i).decode(), float(ms[i])) for i in range(n)]


def osbli_residual_noalloc(params, d_U, d_R, cuda_stream=None):
    """Residual of a device-resident state without any device allocation (see osbli.h)."""
    return _check(None, load().osbli_residual_noalloc(ctypes.byref(params), _ptr(d_U), _ptr(d_R),
                                                      ctypes.c_void_p(cuda_stream or 0)))


def osbli_fp64_peak():
    t = ctypes.c_double()
    _check(None, load().osbli_fp64_peak(ctypes.byref(t)))
    return t.value


def osbli_fp32_peak():
    t = ctypes.c_double()
    _check(None, load().osbli_fp32_peak(ctypes.byref(t)))
    return t.value


def osbli_sensor_set_weights(h, w, threshold):
    w = np.ascontiguousarray(w, dtype=np.float32)
    assert w.size == SENSOR_NPARAM
    return _check(h, load().osbli_sensor_set_weights(h, _ptr(w), float(threshold)))


def osbli_sensor_set_gate(h, flags):
    return _check(h, load().osbli_sensor_set_gate(h, _ptr(flags)))


def osbli_sensor_labels(h, labels):
    return _check(h, load().osbli_sensor_labels(h, _ptr(labels)))


def osbli_sensor_features(h, d_feats):
    return _check(h, load().osbli_sensor_features(h, _ptr(d_feats)))


def osbli_sensor_probs(h, probs):
    return _check(h, load().osbli_sensor_probs(h, _ptr(probs)))


def osbli_mlp_forward(d_feats, n, w, d_probs):
    w = np.ascontiguousarray(w, dtype=np.float32)
    return _check(None, load().osbli_mlp_forward(_ptr(d_feats), int(n), _ptr(w), _ptr(d_probs)))


def osbli_mlp_grad(d_feats, d_labels, n, pos_weight, w):
    w = np.ascontiguousarray(w, dtype=np.float32)
    g = np.zeros(SENSOR_NPARAM, dtype=np.float32)
    loss = ctypes.c_double()
    _check(None, load().osbli_mlp_grad(_ptr(d_feats), _ptr(d_labels), int(n), float(pos_weight),
                                       _ptr(w), _ptr(g), ctypes.byref(loss)))
    return loss.value, g


def osbli_mlp_train(d_feats, d_labels, n, steps, batch, lr, pos_weight, seed, w):
    w = np.array(w, dtype=np.float32, copy=True)
    hist = np.zeros(max(int(steps), 1), dtype=np.float32)
    _check(None, load().osbli_mlp_train(_ptr(d_feats), _ptr(d_labels), int(n), int(steps), int(batch),
                                        float(lr), float(pos_weight), int(seed) & 0xFFFFFFFF,
                                        _ptr(w), _ptr(hist)))
    return w, hist[:int(steps)]


def osbli_last_error(h):
    m = load().osbli_last_error(h)
    return m.decode() if m else ""


def _echeck(e, rc):
    if rc != OSBLI_OK:
        msg = load().osbli_ensemble_last_error(e)
        raise OsbliError(rc, msg.decode() if msg else "")
    return rc


def osbli_ensemble_create(params_list, cuda_stream=None):
    arr = (osbli_params * len(params_list))(*params_list)
    e = ctypes.c_void_p()
    _echeck(None, load().osbli_ensemble_create(len(params_list), arr, ctypes.c_void_p(cuda_stream or 0),
                                               ctypes.byref(e)))
    return e


def osbli_ensemble_destroy(e):
    load().osbli_ensemble_destroy(e)


def osbli_ensemble_set_state(e, p, U):
    return _echeck(e, load().osbli_ensemble_set_state(e, int(p), _ptr(U)))


def osbli_ensemble_get_state(e, p, U):
    return _echeck(e, load().osbli_ensemble_get_state(e, int(p), _ptr(U)))


def osbli_ensemble_member(e, p):
    return load().osbli_ensemble_member(e, int(p))


def osbli_ensemble_step(e, nsteps):
    return _echeck(e, load().osbli_ensemble_step(e, int(nsteps)))


def osbli_ensemble_set_chunk(e, chunk):
    return _echeck(e, load().osbli_ensemble_set_chunk(e, int(chunk)))


def osbli_ensemble_autotune(e, reps=3):
    c = ctypes.c_int()
    ms = ctypes.c_double()
    _echeck(e, load().osbli_ensemble_autotune(e, int(reps), ctypes.byref(c), ctypes.byref(ms)))
    return c.value, ms.value


def osbli_ensemble_launches_per_step(e):
    return load().osbli_ensemble_launches_per_step(e)


def osbli_ensemble_points(e):
    return load().osbli_ensemble_points(e)


def _dcheck(d, rc):
    if rc != OSBLI_OK:
        msg = load().osbli_domain_last_error(d)
        raise OsbliError(rc, msg.decode() if msg else "")
    return rc


def osbli_domain_plan(nz, nslab, periodic):
    """(k0, nzs, lo, hi) lists of the z-split; host only."""
    arrs = [(ctypes.c_int * max(1, nslab))() for _ in range(4)]
    rc = load().osbli_domain_plan(int(nz), int(nslab), int(bool(periodic)), *arrs)
    if rc != OSBLI_OK:
        raise OsbliError(rc, "bad split of %d planes into %d slabs" % (nz, nslab))
    return tuple(list(a)[:nslab] for a in arrs)


def osbli_domain_create(params, nslab, cuda_stream=None):
    d = ctypes.c_void_p()
    _dcheck(None, load().osbli_domain_create(ctypes.byref(params), int(nslab), ctypes.c_void_p(cuda_stream or 0),
                                             ctypes.byref(d)))
    return d


class Domain:
    """One grid split into z-slabs with halo exchanges (osbli_domain_*); same interface as Solver
    for state, stepping and residuals."""

    def __init__(self, cfg, nslab, precision=OSBLI_FP64, cuda_stream=None):
        self.d = None
        self.n = tuple(int(x) for x in cfg["n"])
        self.shape = (5, self.n[2], self.n[1], self.n[0])
        self.d = osbli_domain_create(make_params(cfg, precision), nslab, cuda_stream)
        L = load()
        for (dd, ss), arr in (cfg.get("bdata") or {}).items():
            a = np.ascontiguousarray(arr, dtype=np.float64)
            _dcheck(self.d, L.osbli_domain_set_boundary_data(self.d, int(dd), int(ss), _ptr(a)))

    def close(self):
        if getattr(self, "d", None):
            load().osbli_domain_destroy(self.d)
            self.d = None

    __del__ = close

    def set_state(self, U):
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.shape)
        _dcheck(self.d, load().osbli_domain_set_state(self.d, _ptr(U)))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        _dcheck(self.d, load().osbli_domain_get_state(self.d, _ptr(out)))
        return out

    def step(self, nsteps):
        _dcheck(self.d, load().osbli_domain_step(self.d, int(nsteps)))

    def residual(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        _dcheck(self.d, load().osbli_domain_residual(self.d, _ptr(out)))
        return out

    def slabs(self):
        return load().osbli_domain_slabs(self.d)

    def launches_per_step(self):
        c = ctypes.c_int(0)
        n = load().osbli_domain_launches_per_step(self.d, ctypes.byref(c))
        return n, c.value


class Ensemble:
    """Independent problems advanced together; ``cfgs`` are ``inputs`` problem dicts."""

    def __init__(self, cfgs, precision=OSBLI_MIXED, cuda_stream=None):
        self.e = None
        self.shapes = [(5, int(c["n"][2]), int(c["n"][1]), int(c["n"][0])) for c in cfgs]
        self.e = osbli_ensemble_create([make_params(c, precision) for c in cfgs], cuda_stream)

    def close(self):
        if getattr(self, "e", None):
            osbli_ensemble_destroy(self.e)
            self.e = None

    __del__ = close

    def set_state(self, p, U):
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.shapes[p])
        osbli_ensemble_set_state(self.e, p, U)

    def get_state(self, p, out=None):
        if out is None:
            out = np.empty(self.shapes[p])
        osbli_ensemble_get_state(self.e, p, out)
        return out

    def step(self, nsteps):
        osbli_ensemble_step(self.e, nsteps)

    def set_chunk(self, chunk):
        osbli_ensemble_set_chunk(self.e, chunk)

    def set_persistent(self, on=True, spin_limit=0):
        """One cooperative launch per step() call (on) or one graph per step (off)."""
        _echeck(self.e, load().osbli_ensemble_set_persistent(self.e, int(bool(on)), int(spin_limit)))

    def persistent_grid(self):
        return load().osbli_ensemble_persistent_grid(self.e)

    def autotune(self, reps=3):
        return osbli_ensemble_autotune(self.e, reps)

    def launches_per_step(self):
        return osbli_ensemble_launches_per_step(self.e)

    def points(self):
        return osbli_ensemble_points(self.e)


class Solver:
    """One grid problem on the GPU.  ``cfg`` uses the keys of ``inputs`` problem dicts."""

    def __init__(self, cfg, precision=OSBLI_FP64, cuda_stream=None):
        self.h = None
        self.cfg = cfg
        self.n = tuple(int(x) for x in cfg["n"])
        self.shape = (5, self.n[2], self.n[1], self.n[0])
        self.params = make_params(cfg, precision)
        self.h = osbli_create(self.params, cfg.get("coords"), cuda_stream)
        for (d, s), arr in (cfg.get("bdata") or {}).items():
            osbli_set_boundary_data(self.h, d, s, np.ascontiguousarray(arr, dtype=np.float64))

    def close(self):
        if getattr(self, "h", None):
            osbli_destroy(self.h)
            self.h = None

    __del__ = close

    def set_state(self, U):
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.shape)
        osbli_set_state(self.h, U)

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        osbli_get_state(self.h, out)
        return out

    def step(self, nsteps):
        osbli_rk_step(self.h, nsteps)

    def residual(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        osbli_residual(self.h, out)
        return out

    def diagnostics(self):
        out = np.empty(16)
        osbli_diagnostics(self.h, out)
        return out

    def profile_residual(self, reps=3):
        return osbli_profile_residual(self.h, reps)

    def labels(self):
        lab = np.empty(self.shape[1:], dtype=np.uint8)
        osbli_sensor_labels(self.h, lab)
        return lab

    def set_sensor(self, w, threshold=0.5):
        osbli_sensor_set_weights(self.h, w, threshold)

    def set_gate(self, flags):
        """Fixed cell gate ([nz][ny][nx], nonzero = flagged) in place of the network."""
        f = np.ascontiguousarray(flags, dtype=np.uint8).reshape(self.shape[1:])
        osbli_sensor_set_gate(self.h, f)

    def launches_per_step(self):
        return osbli_launches_per_step(self.h)
