"""CPU FP64 oracle of the OpenSBLI residual / RK-stage path (arXiv:2007.14933).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers.  The oracle is plain C (``osbli_oracle.c``) built with gcc and
loaded through ctypes; it shares no code with the CUDA path and never calls it.

Parity pins (see ``tests/test_oracle_pins.py``): ENO coefficients and optimal weights (5th order and
TENO6) against the polynomial-exactness definition, the printed smoothness indicators against their integral definition
(Eq. 16), WENO/TENO weights on linear and discontinuous data, eigensystem identities, the RK3
amplification polynomial, the exact Riemann solution for Sod, the closed-form viscous and heat-flux
residuals, TGV kinetic-energy pins (initial values and the energy budget over 200 steps), discrete
conservation, the curvilinear order of convergence, the isothermal-wall ghosts on a linear profile,
the Dirichlet and inflow faces against their definition (and a uniform stream through them staying
exact), and the gated convective form against the central and characteristic forms
(``tests/test_oracle_gated.py``).  Without such a pin: the developed flow field of the
shock / boundary-layer box ("parity unpinned"; no reference data exist for it).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "osbli_oracle.c")
_LIB = os.path.join(_HERE, "libosbli_oracle.so")

CENTRAL4, WENO5JS, TENO5, WENO5Z, TENO6 = 0, 1, 2, 3, 4
PERIODIC, ZEROGRAD, WALL, DIRICHLET, INFLOW, ADIABATIC = 0, 1, 2, 3, 4, 5


def build(force=False):
    """Compile the oracle with gcc (no FP contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("gamma", ctypes.c_double), ("Re", ctypes.c_double), ("Pr", ctypes.c_double),
        ("Ma", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("teno_ct", ctypes.c_double),
        ("bc", (ctypes.c_int * 2) * 3),
        ("T_wall", ctypes.c_double),
        ("suth", ctypes.c_double),
        ("h", ctypes.c_double * 3),
        ("L", ctypes.c_double * 3),
        ("coords", ctypes.c_void_p),
        ("bdata", ctypes.c_void_p * 6),
        ("rk", ctypes.c_int),
        ("force", ctypes.c_double * 3),
    ]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(Params)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        for f in (L.orc_set_state, L.orc_get_state):
            f.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_residual.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_residual_ex.argtypes = [ctypes.c_void_p] * 4
        L.orc_set_gate.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]
        L.orc_residual_points.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]
        L.orc_labels.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_step.restype = ctypes.c_int
        L.orc_get_metrics.argtypes = [ctypes.c_void_p] * 4
        L.orc_get_ghosted.argtypes = [ctypes.c_void_p] * 3
        L.orc_eno_coeffs.argtypes = [ctypes.c_int, ctypes.c_void_p]
        L.orc_linear_weights.argtypes = [ctypes.c_void_p]
        L.orc_smoothness5.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_weights5.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                   ctypes.c_void_p]
        L.orc_recon5.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                 ctypes.c_void_p]
        L.orc_recon5.restype = ctypes.c_double
        L.orc_teno6_linear_weights.argtypes = [ctypes.c_void_p]
        L.orc_smoothness_cubic.argtypes = [ctypes.c_void_p]
        L.orc_smoothness_cubic.restype = ctypes.c_double
        L.orc_weights6.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_recon6.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_recon6.restype = ctypes.c_double
        L.orc_flux.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_eigensystem.argtypes = [ctypes.c_double] + [ctypes.c_void_p] * 6
        L.orc_char_flux_1d.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_rk3_linear.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int, _D, _D]
        L.orc_rk_linear.argtypes = [ctypes.c_int] + [ctypes.c_double] * 3 + [ctypes.c_int, _D, _D]
        L.orc_deriv4.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_deriv4.restype = ctypes.c_double
        L.orc_sutherland.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_sutherland.restype = ctypes.c_double
        L.orc_riemann_star.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, _D, _D]
        L.orc_riemann_sample.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_get_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n):
    lib().orc_set_threads(int(n))


def get_threads():
    return lib().orc_get_threads()


class Oracle:
    """A problem instance of the oracle.  ``cfg`` is a dict with the keys of
    ``paper_2007_14933_b300.inputs`` problem descriptions: n, gamma, Re, Pr, Ma, dt, scheme,
    teno_ct, bc, T_wall, suth, h, L, and optionally coords ([3][nz][ny][nx]) and bdata
    ({(d, s): [5][plane]})."""

    def __init__(self, cfg):
        L = lib()
        P = Params()
        n = cfg["n"]
        for d in range(3):
            P.n[d] = int(n[d])
            P.h[d] = float(cfg.get("h", (1.0, 1.0, 1.0))[d])
            P.L[d] = float(cfg.get("L", (0.0, 0.0, 0.0))[d])
            for s in range(2):
                P.bc[d][s] = int(cfg["bc"][d][s])
        P.gamma = cfg.get("gamma", 1.4)
        P.Re = cfg.get("Re", 0.0)
        P.Pr = cfg.get("Pr", 0.72)
        P.Ma = cfg.get("Ma", 1.0)
        P.dt = cfg.get("dt", 0.0)
        P.scheme = int(cfg.get("scheme", TENO5))
        P.teno_ct = cfg.get("teno_ct", 1e-5)
        P.rk = int(cfg.get("rk", 0))
        for q, f in enumerate(cfg.get("force", (0.0, 0.0, 0.0))):
            P.force[q] = float(f)
        P.T_wall = cfg.get("T_wall", 1.0)
        P.suth = cfg.get("suth", 0.0)
        self._keep = []
        coords = cfg.get("coords")
        if coords is not None:
            c = _f64(coords)
            self._keep.append(c)
            P.coords = c.ctypes.data
        for (d, s), arr in (cfg.get("bdata") or {}).items():
            a = _f64(arr)
            self._keep.append(a)
            P.bdata[2 * d + s] = a.ctypes.data
        self.n = tuple(int(x) for x in n)
        self.shape = (5, self.n[2], self.n[1], self.n[0])
        self._h = L.orc_create(ctypes.byref(P))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def set_state(self, U):
        U = _f64(U).reshape(self.shape)
        lib().orc_set_state(self._h, _p(U))

    def get_state(self):
        U = np.empty(self.shape)
        lib().orc_get_state(self._h, _p(U))
        return U

    def residual(self, with_margin=False, with_jump_margin=False):
        """R(U).  with_margin: also the per-node smallest TENO |chi - C_T|/C_T; with_jump_margin
        (gated form): also the per-node smallest |ratio/jump - 1| of its strong-jump tests."""
        R = np.empty(self.shape)
        m = np.empty(self.shape[1:]) if with_margin else None
        jm = np.empty(self.shape[1:]) if with_jump_margin else None
        lib().orc_residual_ex(self._h, _p(R), _p(m) if with_margin else None,
                              _p(jm) if with_jump_margin else None)
        out = (R,) + ((m,) if with_margin else ()) + ((jm,) if with_jump_margin else ())
        return out if len(out) > 1 else R

    def set_gate(self, gate, jump=1.5):
        """Gated convective form: gate [nz][ny][nx] (nonzero = the cell's interfaces take the
        characteristic flux), interfaces with a strong jump (ratio > jump) too, the others the
        central 4th-order interface flux.  None returns to the plain scheme."""
        if gate is None:
            lib().orc_set_gate(self._h, None, float(jump))
            return
        g = np.ascontiguousarray(gate, dtype=np.uint8).reshape(self.shape[1:])
        lib().orc_set_gate(self._h, _p(g), float(jump))

    def residual_points(self, ijk, with_margin=False):
        ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        R = np.empty((ijk.shape[0], 5))
        m = np.empty(ijk.shape[0])
        lib().orc_residual_points(self._h, ijk.shape[0], _p(ijk), _p(R), _p(m))
        return (R, m) if with_margin else R

    def labels(self):
        """TENO cut-off labels of the current state ([nz][ny][nx] uint8)."""
        lab = np.empty(self.shape[1:], dtype=np.uint8)
        lib().orc_labels(self._h, _p(lab))
        return lab

    def step(self, nsteps):
        rc = lib().orc_step(self._h, int(nsteps))
        if rc != 0:
            raise FloatingPointError("oracle state became non-finite")

    def metrics(self):
        S = np.empty((9,) + self.shape[1:])
        J = np.empty(self.shape[1:])
        sh = np.empty(3)
        lib().orc_get_metrics(self._h, _p(S), _p(J), _p(sh))
        return S.reshape((3, 3) + self.shape[1:]), J, sh

    def ghosted(self):
        np_ = np.zeros(3, dtype=np.int32)
        g = [3 if x > 1 else 0 for x in self.n]
        tot = 5 * np.prod([self.n[d] + 2 * g[d] for d in range(3)])
        Ug = np.empty(tot)
        lib().orc_get_ghosted(self._h, _p(Ug), _p(np_))
        return Ug.reshape(5, np_[2], np_[1], np_[0])


# ---- unit-level entry points used by the pins -------------------------------------------------

def eno_coeffs(k):
    c = np.empty(k * k)
    lib().orc_eno_coeffs(k, _p(c))
    return c.reshape(k, k)


def linear_weights():
    d = np.empty(3)
    lib().orc_linear_weights(_p(d))
    return d


def smoothness5(f):
    f = _f64(f)
    b = np.empty(3)
    lib().orc_smoothness5(_p(f), _p(b))
    return b


def weights5(beta, scheme, ct=1e-5):
    beta = _f64(beta)
    w = np.empty(3)
    m = np.empty(1)
    lib().orc_weights5(_p(beta), int(scheme), float(ct), _p(w), _p(m))
    return w, float(m[0])


def recon5(f, scheme, ct=1e-5):
    f = _f64(f)
    w = np.empty(3)
    m = np.empty(1)
    v = lib().orc_recon5(_p(f), int(scheme), float(ct), _p(w), _p(m))
    return v, w


def teno6_linear_weights():
    d = np.empty(4)
    lib().orc_teno6_linear_weights(_p(d))
    return d


def smoothness_cubic(g):
    return lib().orc_smoothness_cubic(_p(_f64(g)))


def weights6(beta, ct=1e-5):
    beta = _f64(beta)
    w = np.empty(4)
    m = np.empty(1)
    lib().orc_weights6(_p(beta), float(ct), _p(w), _p(m))
    return w, float(m[0])


def recon6(f, ct=1e-5):
    f = _f64(f)
    w = np.empty(4)
    m = np.empty(1)
    v = lib().orc_recon6(_p(f), float(ct), _p(w), _p(m))
    return v, w


def flux(gamma, U, S):
    U = _f64(U)
    S = _f64(S)
    F = np.empty(5)
    lib().orc_flux(gamma, _p(U), _p(S), _p(F))
    return F


def eigensystem(gamma, UL, UR, n):
    UL, UR, n = _f64(UL), _f64(UR), _f64(n)
    R = np.empty(25)
    Lm = np.empty(25)
    lam = np.empty(5)
    lib().orc_eigensystem(gamma, _p(UL), _p(UR), _p(n), _p(R), _p(Lm), _p(lam))
    return R.reshape(5, 5), Lm.reshape(5, 5), lam


def char_flux_1d(gamma, scheme, ct, U6, S):
    U6 = _f64(U6).reshape(6, 5)
    S = _f64(S)
    F = np.empty(5)
    lib().orc_char_flux_1d(gamma, int(scheme), float(ct), _p(U6), _p(S), _p(F))
    return F


def rk3_linear(lam, dt, nsteps, y0=1.0 + 0j):
    return rk_linear(0, lam, dt, nsteps, y0)


def rk_linear(rk, lam, dt, nsteps, y0=1.0 + 0j):
    yr = ctypes.c_double(y0.real)
    yi = ctypes.c_double(y0.imag)
    lib().orc_rk_linear(int(rk), lam.real, lam.imag, dt, int(nsteps), ctypes.byref(yr), ctypes.byref(yi))
    return complex(yr.value, yi.value)


def deriv4(v, i, periodic):
    v = _f64(v)
    return lib().orc_deriv4(_p(v), v.size, int(i), int(periodic))


def sutherland(T, suth):
    return lib().orc_sutherland(float(T), float(suth))


def riemann_star(gamma, WL, WR):
    ps = ctypes.c_double()
    us = ctypes.c_double()
    lib().orc_riemann_star(gamma, _p(_f64(WL)), _p(_f64(WR)), ctypes.byref(ps), ctypes.byref(us))
    return ps.value, us.value


def riemann_sample(gamma, WL, WR, x0, t, x):
    x = _f64(x)
    r, u, p = np.empty_like(x), np.empty_like(x), np.empty_like(x)
    lib().orc_riemann_sample(gamma, _p(_f64(WL)), _p(_f64(WR)), x0, t, x.size, _p(x), _p(r),
                             _p(u), _p(p))
    return r, u, p
