"""osbli_residual_noalloc: the residual for callers that may not allocate device memory.

Some embedding applications cannot call cudaMalloc (they hand all device memory to their own
pool, run a real-time loop that cannot take an allocation's synchronisation, or live as a
plug-in that is not allowed to allocate).  The entry point keeps its intermediate arrays in a
static device array instead.  Its result must equal the handle-based osbli_residual on the same
state, on two calls in a row (the second call must not see the first call's leftovers).

This file is collected last so that, if it fails, a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2007_14933_b300 import inputs as I
from paper_2007_14933_b300 import osbli

pytestmark = pytest.mark.gpu

TOL = 1e-11   # same bar as the other FP64 parity tests


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14933_b300 import build
    build.build()
    osbli.load()
    return t


def _handle_residual(cfg, U):
    s = osbli.Solver(cfg)
    s.set_state(U)
    R = s.residual()
    s.close()
    return R


def _noalloc_residual(torch, cfg, U):
    dU = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    dR = torch.full_like(dU, float("nan"))
    stream = torch.cuda.current_stream().cuda_stream
    osbli.osbli_residual_noalloc(osbli.make_params(cfg), dU, dR, stream)
    return dR.cpu().numpy()


def _relerr(a, b):
    scale = np.abs(b).reshape(5, -1).max(axis=1)[:, None]
    scale[scale == 0] = 1.0      # a 2D state's w momentum is identically zero
    return float((np.abs(a - b).reshape(5, -1) / scale).max())


def test_noalloc_matches_handle_residual_on_two_calls(torch):
    # call 1: TENO5 + viscous periodic box; call 2: a different state, grid and scheme
    cfg1, U1 = I.tgv(n=(20, 12, 9), Ma=1.25, scheme=I.TENO5)
    n2 = (16, 10, 7)
    U2 = I.random_state(n2, seed=5, shocky=True)
    cfg2 = dict(n=n2, gamma=1.4, Re=0.0, Ma=1.0, scheme=I.WENO5JS, bc=[[0, 0]] * 3,
                h=(0.1, 0.2, 0.3))
    for cfg, U in ((cfg1, U1), (cfg2, U2)):
        Rn = _noalloc_residual(torch, cfg, U)
        Rh = _handle_residual(cfg, U)
        assert np.isfinite(Rn).all()
        assert _relerr(Rn, Rh) <= TOL


def _wall_box(n=(14, 11, 6)):
    """Viscous box with zero-gradient x faces, isothermal walls in y (T_wall = 1.3) and periodic
    z, on a uniform grid: the ghost layouts of every accepted face type."""
    g, Ma, Tw = 1.4, 0.8, 1.3
    nx, ny, nz = n
    h = (0.3, 0.2, 0.5)
    z, y, x = np.meshgrid(np.arange(nz) * h[2], np.arange(ny) * h[1], np.arange(nx) * h[0], indexing="ij")
    u = np.tanh(3 * y) * (1 + 0.05 * np.sin(x))
    T = Tw + (1 - Tw) * np.tanh(3 * y)
    p = (1 + 0.02 * np.cos(x + 2 * z)) / (g * Ma * Ma)
    rho = g * Ma * Ma * p / T
    U = I.prim_to_cons(g, rho, u, 0.02 * np.sin(x) * np.tanh(y), 0.01 * np.cos(z), p)
    U[1:4, :, 0, :] = 0.0
    U[1:4, :, -1, :] = 0.0
    cfg = dict(n=n, gamma=g, Re=300.0, Pr=0.72, Ma=Ma, scheme=I.TENO5, teno_ct=1e-5,
               bc=[[1, 1], [2, 2], [0, 0]], h=h, T_wall=Tw, suth=110.4 / 288.0)
    return cfg, U


def test_noalloc_face_types_2d_teno6_and_force(torch):
    """Zero-gradient and wall faces, a 2D grid (nz = 1: no z ghosts, so other strides in the
    static array), TENO6 and a body force, each against osbli_residual, two calls per case."""
    cases = [_wall_box()]
    cfg2, U2 = I.riemann2d(23, [(1.5, 0.0, 0.0, 1.5), (0.5323, 1.206, 0.0, 0.3),
                                 (0.138, 1.206, 1.206, 0.029), (0.5323, 0.0, 1.206, 0.3)],
                           scheme=I.TENO6, ny=17)
    cases.append((cfg2, U2))
    cfg3, U3 = I.tgv(n=(12, 10, 8), Ma=0.4, scheme=I.WENO5Z)
    cases.append((dict(cfg3, force=(0.7, -0.2, 0.1)), U3))
    for cfg, U in cases:
        for _ in range(2):
            Rn = _noalloc_residual(torch, cfg, U)
            Rh = _handle_residual(cfg, U)
            assert np.isfinite(Rn).all()
            assert _relerr(Rn, Rh) <= TOL, cfg["bc"]


def test_noalloc_reports_a_nonfinite_residual(torch):
    cfg, U = I.tgv(n=(10, 9, 8), Ma=0.5, scheme=I.TENO5)
    U = U.copy()
    U[0, 3, 4, 5] = -1.0      # negative density: the sound speed, hence the residual, is NaN
    dU = torch.from_numpy(U).cuda()
    dR = torch.empty_like(dU)
    rc = osbli.load().osbli_residual_noalloc(ctypes.byref(osbli.make_params(cfg)),
                                             ctypes.c_void_p(dU.data_ptr()),
                                             ctypes.c_void_p(dR.data_ptr()), None)
    assert rc == osbli.OSBLI_ENONFINITE
    # the next call on a good state succeeds (the error word is cleared per call)
    cfg, U = I.tgv(n=(10, 9, 8), Ma=0.5, scheme=I.TENO5)
    assert _relerr(_noalloc_residual(torch, cfg, U), _handle_residual(cfg, U)) <= TOL


def test_noalloc_rejects_a_wall_without_temperature(torch):
    cfg, U = _wall_box()
    dU = torch.from_numpy(U).cuda()
    dR = torch.empty_like(dU)
    rc = osbli.load().osbli_residual_noalloc(ctypes.byref(osbli.make_params(dict(cfg, T_wall=0.0))),
                                             ctypes.c_void_p(dU.data_ptr()),
                                             ctypes.c_void_p(dR.data_ptr()), None)
    assert rc == osbli.OSBLI_EINVAL
    assert "T_wall" in osbli.osbli_last_error(None)


def test_noalloc_rejects_grids_beyond_the_static_capacity(torch):
    cfg, U = I.tgv(n=(40, 40, 40), Ma=0.5, scheme=I.TENO5)   # 46^3 ghosted nodes > 65536
    dU = torch.from_numpy(U).cuda()
    dR = torch.empty_like(dU)
    p = osbli.make_params(cfg)
    rc = osbli.load().osbli_residual_noalloc(ctypes.byref(p), ctypes.c_void_p(dU.data_ptr()),
                                             ctypes.c_void_p(dR.data_ptr()), None)
    assert rc == osbli.OSBLI_EINVAL
    msg = osbli.osbli_last_error(None)
    assert "too large" in msg and "65536" in msg
