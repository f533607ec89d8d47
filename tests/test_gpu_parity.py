"""GPU (libosbli, through the C ABI) against the CPU oracle, element by element.

Points where the oracle itself is ill-conditioned (its residual moves by more than 1e-11 under a
1e-15 relative perturbation of the state; found with WENO-Z on exactly symmetric TGV data) are
likewise checked with the loose bound only.

Tolerance (plain FP64 path): max over variables v and points of |X_gpu - X_oracle| divided by
max over points |X_oracle,v| must be <= 1e-11 (the three momentum components share one scale,
the largest of their maxima, so that a component that vanishes in exact arithmetic -- spanwise
momentum of a 2D flow -- is judged against the momentum, not against its own rounding noise), for single residual evaluations and after
multi-step runs.  For TENO5 and TENO6 a stencil cut-off decision delta_r = [chi_r >= C_T] whose chi_r
lies within rounding of C_T may legitimately differ between two correct FP64 evaluations; points
whose oracle margin |chi - C_T|/C_T is below 1e-9 are checked separately (bounded deviation)
instead of at 1e-11.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2007_14933_b300 import inputs as I
from paper_2007_14933_b300 import osbli

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14933_b300 import build
    build.build()
    osbli.load()


def relerr(a, b, mask=None):
    a = a.reshape(5, -1)
    b = b.reshape(5, -1)
    scale = np.abs(b).max(axis=1, keepdims=True)
    scale[1:4] = scale[1:4].max()       # momentum components share the momentum scale
    scale[scale == 0] = 1.0
    e = np.abs(a - b) / scale
    if mask is not None:
        e = e[:, mask.reshape(-1)]
    return float(e.max()) if e.size else 0.0


def residual_pair(cfg, U):
    s = osbli.Solver(cfg)
    s.set_state(U)
    Rg = s.residual()
    o = O.Oracle(cfg)
    o.set_state(U)
    Ro, margin = o.residual(with_margin=True)
    return Rg, Ro, margin


def sensitive_points(cfg, U, Ro):
    """Points whose oracle residual moves by more than 1e-11 (relative) when the state is perturbed
    by one part in 1e15: two correct FP64 evaluations may legitimately differ there.  WENO-Z's
    weights (Eq. 22, eps = 1e-16) are ill-conditioned at such points of exactly symmetric data."""
    rng = np.random.default_rng(0)
    o = O.Oracle(cfg)
    o.set_state(U * (1 + 1e-15 * rng.standard_normal(U.shape)))
    R1 = o.residual()
    d = np.abs(R1 - Ro).reshape(5, -1)
    scale = np.abs(Ro).reshape(5, -1).max(axis=1)
    scale[1:4] = scale[1:4].max()
    return (d / scale[:, None]).max(axis=0).reshape(Ro.shape[1:]) > 1e-11


def check_residual(cfg, U):
    Rg, Ro, margin = residual_pair(cfg, U)
    safe = margin > 1e-9
    if cfg.get("scheme") == I.WENO5Z:
        safe &= ~sensitive_points(cfg, U, Ro)
    assert relerr(Rg, Ro, safe) <= TOL
    if (~safe).any():   # ambiguous TENO cut-offs: still bounded
        assert relerr(Rg, Ro) < 1e-3
    return Rg, Ro


def wall_box(n=(16, 12, 4), scheme=I.TENO5, skew=0.0):
    """Small box with every non-periodic boundary type: inflow / zero-gradient in x, isothermal
    wall / Dirichlet in y (tanh-stretched), periodic z, Sutherland viscosity.  skew = 0 keeps the
    grid rectilinear (Cartesian kernels with per-line factors); skew > 0 shears the grid lines
    (x shifted with y and z) so that the general curvilinear kernels run."""
    g, Ma = 1.4, 2.0
    nx, ny, nz = n
    Lx, Ly, Lz = 10.0, 4.0, 2.0
    x = np.linspace(0, Lx, nx)
    j = np.arange(ny)
    y = Ly * (1 - np.tanh(1.5 * (1 - j / (ny - 1))) / np.tanh(1.5))
    z = np.arange(nz) * Lz / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    coords = np.stack([X + skew * np.sin(math.pi * Y / Ly) * (1 + 0.3 * np.cos(2 * math.pi * Z / Lz)), Y, Z])
    Tw = 1.7
    eta = Y / 1.0
    u = np.tanh(2 * eta) * (1 + 0.02 * np.sin(2 * math.pi * Z / Lz))
    T = Tw + (1 - Tw) * np.tanh(2 * eta)
    p = np.full_like(u, 1.0 / (g * Ma * Ma)) * (1 + 0.01 * np.sin(X))
    rho = g * Ma * Ma * p / T
    v = 0.01 * np.tanh(eta) * np.cos(X)
    w = 0.01 * np.sin(2 * math.pi * Z / Lz) * np.tanh(eta)
    U = I.prim_to_cons(g, rho, u, v, w, p)
    U[1:4, :, 0, :] = 0.0
    U[4, :, 0, :] = U[0, :, 0, :] * Tw / (Ma * Ma * g * (g - 1))
    inflow = np.zeros((5, nz, ny))
    inflow[1] = u[:, :, 0]
    inflow[2] = v[:, :, 0]
    inflow[3] = w[:, :, 0]
    inflow[4] = T[:, :, 0]
    top = np.zeros((5, nz, nx))
    top[0] = rho[:, -1, :] * 1.05
    top[1] = u[:, -1, :]
    top[2] = -0.05
    top[3] = 0.0
    top[4] = p[:, -1, :] * 1.1
    cfg = dict(n=n, gamma=g, Re=500.0, Pr=0.72, Ma=Ma, dt=2e-3, scheme=scheme, teno_ct=1e-5,
               bc=[[I.INFLOW, I.ZEROGRAD], [I.WALL, I.DIRICHLET], [I.PERIODIC, I.PERIODIC]],
               T_wall=Tw, suth=110.4 / 288.0, h=(1, 1, 1), L=(0, 0, Lz), coords=coords,
               bdata={(0, 0): inflow.reshape(5, -1), (1, 1): top.reshape(5, -1)})
    return cfg, U


# ------------------------------------------------------------------------ single residual
def test_residual_tgv_central_viscous():
    cfg, U = I.tgv(16, Ma=0.1, scheme=I.CENTRAL4)
    check_residual(cfg, U)


@pytest.mark.parametrize("scheme", [I.TENO5, I.WENO5JS, I.WENO5Z, I.TENO6])
def test_residual_tgv_characteristic_viscous_ragged(scheme):
    cfg, U = I.tgv(n=(20, 12, 9), Ma=1.25, scheme=scheme)
    check_residual(cfg, U)


@pytest.mark.parametrize("scheme", [I.TENO5, I.WENO5JS, I.WENO5Z, I.TENO6])
def test_residual_shocky_random_state(scheme):
    n = (13, 9, 7)
    U = I.random_state(n, seed=3, shocky=True)
    cfg = dict(n=n, gamma=1.4, Re=0.0, Ma=1.0, scheme=scheme, teno_ct=1e-5,
               bc=[[0, 0]] * 3, h=(0.1, 0.2, 0.3))
    check_residual(cfg, U)


def test_residual_sod():
    cfg, U, _ = I.sod()
    check_residual(cfg, U)


@pytest.mark.parametrize("scheme", [I.TENO5, I.WENO5JS, I.CENTRAL4, I.WENO5Z, I.TENO6])
def test_residual_curvilinear_euler_wave(scheme):
    cfg, U = I.euler_wave(24, scheme=scheme)
    check_residual(cfg, U)


@pytest.mark.parametrize("skew", [0.0, 0.4])
@pytest.mark.parametrize("scheme", [I.TENO5, I.CENTRAL4, I.TENO6])
def test_residual_walls_inflow_dirichlet(scheme, skew):
    cfg, U = wall_box(scheme=scheme, skew=skew)
    check_residual(cfg, U)


# ------------------------------------------------------------------------ multi-step runs
def run_pair(cfg, U, nsteps):
    s = osbli.Solver(cfg)
    s.set_state(U)
    s.step(nsteps)
    Ug = s.get_state()
    o = O.Oracle(cfg)
    o.set_state(U)
    o.step(nsteps)
    return Ug, o.get_state()


def test_sod_800_steps_matches_oracle_and_exact():
    cfg, U, x = I.sod()
    Ug, Uo = run_pair(cfg, U, 800)
    assert relerr(Ug, Uo) <= TOL
    r, _, _ = O.riemann_sample(1.4, [1, 0, 1], [0.125, 0, 0.1], 0.5, 0.2, x)
    assert np.abs(Ug[0, 0, 0] - r).mean() < 4e-3


def test_tgv_central_100_steps():
    cfg, U = I.tgv(16, Ma=0.1, scheme=I.CENTRAL4)
    Ug, Uo = run_pair(cfg, U, 100)
    assert relerr(Ug, Uo) <= TOL


def test_tgv_central_64_200_steps_and_kinetic_energy():
    """The C2 configuration as stated: TGV 64^3, Ma 0.1, Re 1600, 4th-order central + viscous,
    200 RK3 steps at CFL 0.5 (t = 0.32); the state matches the oracle at the FP64 bar and the
    kinetic-energy history (the GPU's own diagnostic, every 50 steps) the oracle's to 1e-12."""
    import os
    O.set_threads(len(os.sched_getaffinity(0)))
    cfg, U = I.tgv(64, Ma=0.1, scheme=I.CENTRAL4)
    s = osbli.Solver(cfg)
    s.set_state(U)
    o = O.Oracle(cfg)
    o.set_state(U)
    for _ in range(4):
        s.step(50)
        o.step(50)
        Uo = o.get_state()
        ke_o = float((0.5 * (Uo[1] ** 2 + Uo[2] ** 2 + Uo[3] ** 2) / Uo[0]).mean())
        assert abs(s.diagnostics()[5] - ke_o) <= 1e-12 * ke_o
    Ug = s.get_state()
    s.close()
    assert relerr(Ug, Uo) <= TOL


def test_tgv_teno_100_steps():
    cfg, U = I.tgv(12, Ma=1.25, scheme=I.TENO5)
    Ug, Uo = run_pair(cfg, U, 100)
    assert relerr(Ug, Uo) <= TOL


def test_tgv_teno6_100_steps():
    cfg, U = I.tgv(12, Ma=1.25, scheme=I.TENO6)
    Ug, Uo = run_pair(cfg, U, 100)
    assert relerr(Ug, Uo) <= TOL


def test_sod_teno6_800_steps_matches_oracle_and_exact():
    cfg, U, x = I.sod(scheme=I.TENO6)
    Ug, Uo = run_pair(cfg, U, 800)
    assert relerr(Ug, Uo) <= TOL
    r, _, _ = O.riemann_sample(1.4, [1, 0, 1], [0.125, 0, 0.1], 0.5, 0.2, x)
    assert np.abs(Ug[0, 0, 0] - r).mean() < 4e-3


def test_euler_wave_teno_100_steps():
    cfg, U = I.euler_wave(32, scheme=I.TENO5)
    Ug, Uo = run_pair(cfg, U, 100)
    assert relerr(Ug, Uo) <= TOL


@pytest.mark.parametrize("skew", [0.0, 0.4])
def test_walls_20_steps(skew):
    cfg, U = wall_box(skew=skew)
    Ug, Uo = run_pair(cfg, U, 20)
    assert relerr(Ug, Uo) <= TOL


# ------------------------------------------------------------------------ full-size samples
def _sample_points(n, count, seed):
    rng = np.random.default_rng(seed)
    pts = np.stack([rng.integers(0, n[d], size=count) for d in range(3)], axis=1)
    corners = np.array([[i, j, k] for i in (0, 1, n[0] - 1) for j in (0, n[1] - 2, n[1] - 1)
                        for k in (0, n[2] - 1)])
    return np.concatenate([pts, corners]).astype(np.int32)


@pytest.mark.parametrize("which", ["tgv256_teno", "tgv128_central"])
def test_full_size_residual_sampled(which):
    if which == "tgv256_teno":
        cfg, U = I.tgv(256, Ma=1.25, scheme=I.TENO5)
    else:
        cfg, U = I.tgv(128, Ma=0.1, scheme=I.CENTRAL4)
    s = osbli.Solver(cfg)
    s.set_state(U)
    Rg = s.residual()
    o = O.Oracle(cfg)
    o.set_state(U)
    pts = _sample_points(cfg["n"], 300, 7)
    Ro, margin = o.residual_points(pts, with_margin=True)
    Rgs = Rg[:, pts[:, 2], pts[:, 1], pts[:, 0]].T
    scale = np.abs(Rg).reshape(5, -1).max(axis=1)
    err = np.abs(Rgs - Ro) / scale
    safe = margin > 1e-9
    assert err[safe].max() <= TOL


def test_full_size_tgv256_teno_steps_conserve():
    cfg, U = I.tgv(256, Ma=1.25, scheme=I.TENO5)
    s = osbli.Solver(cfg)
    s.set_state(U)
    d0 = s.diagnostics()
    s.step(5)
    d1 = s.diagnostics()
    scale = np.abs(U).reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(d1[:5] - d0[:5]) <= 1e-12 * scale + 1e-9)
    assert d1[5] < d0[5]          # kinetic energy decays
    assert np.isfinite(s.get_state()).all()


# ------------------------------------------------------------------------ determinism, errors
def test_steps_are_deterministic_and_graph_replay_splits():
    cfg, U = I.tgv(n=(16, 12, 8), Ma=1.25, scheme=I.TENO5)
    a = osbli.Solver(cfg)
    a.set_state(U)
    a.step(10)
    b = osbli.Solver(cfg)
    b.set_state(U)
    b.step(4)
    b.step(6)
    np.testing.assert_array_equal(a.get_state(), b.get_state())
    c = osbli.Solver(cfg)
    mid = osbli.Solver(cfg)
    mid.set_state(U)
    mid.step(3)
    c.set_state(mid.get_state())
    c.step(7)
    np.testing.assert_array_equal(a.get_state(), c.get_state())


def test_nonfinite_state_is_reported():
    cfg, U = I.tgv(12, Ma=0.5, scheme=I.TENO5)
    U = U.copy()
    U[4, 3, 4, 5] = np.nan
    s = osbli.Solver(cfg)
    s.set_state(U)
    with pytest.raises(osbli.OsbliError) as e:
        s.step(1)
    assert e.value.code == osbli.OSBLI_ENONFINITE


def test_step_before_set_state_is_rejected():
    cfg, U = I.tgv(12, Ma=0.5, scheme=I.TENO5)
    s = osbli.Solver(cfg)
    with pytest.raises(osbli.OsbliError) as e:
        s.step(1)
    assert e.value.code == osbli.OSBLI_ESTATE


def test_torch_device_buffers_roundtrip():
    import torch
    cfg, U = I.tgv(n=(10, 8, 6), Ma=0.5, scheme=I.TENO5)
    s = osbli.Solver(cfg, cuda_stream=torch.cuda.current_stream().cuda_stream)
    Ud = torch.from_numpy(U).cuda()
    s.set_state(Ud)
    out = torch.empty_like(Ud)
    osbli.osbli_get_state(s.h, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), U)


@pytest.mark.parametrize("scheme", [I.TENO5, I.CENTRAL4])
def test_rk4_five_stage_steps(scheme):
    """The 5-stage 4th-order low-storage integrator (rk = 1) against the oracle's."""
    cfg, U = I.tgv(12, Ma=1.25 if scheme != I.CENTRAL4 else 0.1, scheme=scheme)
    cfg = dict(cfg, rk=1)
    Ug, Uo = run_pair(cfg, U, 30)
    assert relerr(Ug, Uo) <= TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ssprk3_steps(precision):
    """The 3rd-order SSP integrator (rk = 2, convex form) against the oracle's: Sod with walls of
    zero-gradient faces (boundary nodes) and the TENO5 TGV; the mixed path by relative L2."""
    for cfg, U, steps in [(*I.sod()[:2], 200), (*I.tgv(12, Ma=1.25, scheme=I.TENO5), 30)]:
        cfg = dict(cfg, rk=2)
        if precision == "fp64":
            Ug, Uo = run_pair(cfg, U, steps)
            assert relerr(Ug, Uo) <= TOL
        else:
            s = osbli.Solver(cfg, precision=osbli.OSBLI_MIXED)
            s.set_state(U)
            s.step(steps)
            Ug = s.get_state()
            s.close()
            o = O.Oracle(cfg)
            o.set_state(U)
            o.step(steps)
            Uo = o.get_state()
            a, b = Ug.reshape(5, -1), Uo.reshape(5, -1)
            nb = [np.linalg.norm(b[v]) for v in range(5)]
            nb[1] = nb[2] = nb[3] = max(nb[1:4])
            assert max(np.linalg.norm(a[v] - b[v]) / nb[v] for v in range(5) if nb[v] > 0) <= 1e-5


def test_laminar_channel_adiabatic_wall_and_forcing():
    """Sec. 5.4 channel (isothermal + adiabatic walls, unit body force): the analytic state stays
    steady on the GPU (its residual is rounding noise on both sides), and from a perturbed state
    the residual and 30 steps match the oracle."""
    cfg, U, y = I.laminar_channel()
    s = osbli.Solver(cfg)
    s.set_state(U)
    s.step(30)
    Ug = s.get_state()
    s.close()
    for v in (0, 1, 4):
        assert np.abs(Ug[v] - U[v]).max() <= 1e-12 * np.abs(U[v]).max()
    g = 1.4
    Y = y[None, :, None]
    X = (np.arange(cfg["n"][0]) * 2 * math.pi / cfg["n"][0])[None, None, :]
    rho = U[0] * (1 + 1e-3 * np.sin(X) * (1 - Y ** 2))
    u = U[1] / U[0] * (1 + 1e-2 * np.cos(2 * X))
    v = 0.05 * np.sin(X) * (1 - Y ** 2)
    p = (g - 1) * (U[4] - 0.5 * U[1] ** 2 / U[0]) * (1 + 1e-3 * np.cos(X + Y))
    V = I.prim_to_cons(g, rho, u, v, np.zeros_like(u), p)
    check_residual(cfg, V)
    Ug, Uo = run_pair(cfg, V, 30)
    assert relerr(Ug, Uo) <= TOL
