"""Seeded / analytic problem set-ups shared by the CUDA path and the oracle.

This module holds problem descriptions, grids and initial states only: none of the method's
arithmetic (no flux, reconstruction, eigensystem, viscous term or time update).  A problem is a
plain dict:

    n        interior points (nx, ny, nz); 1 marks an inactive direction
    gamma, Re, Pr, Ma   (Re <= 0: inviscid)
    dt       fixed time step
    scheme   0 central 4th order, 1 WENO5-JS, 2 TENO5 (characteristic, Roe average)
    teno_ct  TENO cut-off C_T
    bc       bc[d][s]: 0 periodic, 1 zero-gradient, 2 isothermal wall, 3 Dirichlet, 4 inflow
    T_wall, suth (T_s/T_ref of Sutherland's law, <= 0: mu = 1)
    h, L     uniform spacings / periods
    coords   optional [3][nz][ny][nx] node coordinates (curvilinear grids)
    bdata    optional {(d, s): [5][plane]} face data for Dirichlet / inflow faces

Workloads (paper sections in brackets):
    sod()          1D Sod shock tube [Sec. 5.1], WENO5-JS, N=400, dt=2.5e-4, 800 steps to t=0.2
    tgv()          3D Taylor-Green vortex [Sec. 7], periodic cube of side 2 pi; central 4th order +
                   viscous at Ma 0.1 (64^3, 128^3) or TENO5 + viscous at Ma 1.25 (256^3)
    euler_wave()   2D density wave on the sinusoidal curvilinear grid [Sec. 5.3, Eqs. 47-50]
    random_state() seeded smooth/perturbed states for parity tests
"""
import math

import numpy as np

CENTRAL4, WENO5JS, TENO5 = 0, 1, 2
PERIODIC, ZEROGRAD, WALL, DIRICHLET, INFLOW = 0, 1, 2, 3, 4


def prim_to_cons(gamma, rho, u, v, w, p):
    """Conserved variables (rho, rho u, rho v, rho w, rho E) from primitives (definition of E)."""
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E]).astype(np.float64)


def _base(n, **kw):
    cfg = dict(n=tuple(n), gamma=1.4, Re=0.0, Pr=0.72, Ma=1.0, dt=0.0, scheme=TENO5, teno_ct=1e-5,
               bc=[[PERIODIC, PERIODIC]] * 3, T_wall=1.0, suth=0.0, h=(1.0, 1.0, 1.0),
               L=(0.0, 0.0, 0.0), coords=None, bdata=None)
    cfg.update(kw)
    return cfg


def cfl_dt(cfg, U, cfl):
    """Fixed time step from a CFL number on the initial state: dt = CFL / max sum_d (|u_d|+a)/h_d."""
    g = cfg["gamma"]
    rho = U[0]
    u = [U[1] / rho, U[2] / rho, U[3] / rho]
    p = (g - 1.0) * (U[4] - 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2))
    a = np.sqrt(g * p / rho)
    s = np.zeros_like(rho)
    for d in range(3):
        if cfg["n"][d] > 1:
            s = s + (np.abs(u[d]) + a) / cfg["h"][d]
    return float(cfl / s.max())


# ---------------------------------------------------------------------------------------------
def sod(N=400, scheme=WENO5JS, dt=2.5e-4):
    """Sod shock tube: (rho,u,p) = (1,0,1) for x < 0.5 and (0.125,0,0.1) otherwise, nodes at
    x_i = (i + 1/2)/N, zero-gradient ends, inviscid."""
    cfg = _base((N, 1, 1), scheme=scheme, dt=dt, h=(1.0 / N, 1.0, 1.0),
                bc=[[ZEROGRAD, ZEROGRAD], [PERIODIC, PERIODIC], [PERIODIC, PERIODIC]])
    x = (np.arange(N) + 0.5) / N
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    z = np.zeros(N)
    U = prim_to_cons(cfg["gamma"], rho, z, z, z, p).reshape(5, 1, 1, N)
    return cfg, U, x


def tgv(N=64, Ma=0.1, Re=1600.0, scheme=CENTRAL4, cfl=0.5, Pr=0.72, n=None):
    """Taylor-Green vortex on [0, 2 pi)^3: u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    p = 1/(gamma Ma^2) + (cos 2x + cos 2y)(cos 2z + 2)/16, T = 1 (rho = gamma Ma^2 p), mu = 1."""
    n = tuple(n) if n is not None else (N, N, N)
    h = tuple(2.0 * math.pi / m for m in n)
    cfg = _base(n, scheme=scheme, Re=Re, Pr=Pr, Ma=Ma, h=h,
                L=(2.0 * math.pi,) * 3)
    x = np.arange(n[0]) * h[0]
    y = np.arange(n[1]) * h[1]
    zc = np.arange(n[2]) * h[2]
    Z, Y, X = np.meshgrid(zc, y, x, indexing="ij")
    g = cfg["gamma"]
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p = 1.0 / (g * Ma * Ma) + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    rho = g * Ma * Ma * p
    U = prim_to_cons(g, rho, u, v, w, p)
    cfg["dt"] = cfl_dt(cfg, U, cfl)
    return cfg, U


def euler_wave_grid(N, A=0.04, Lx=2.0, Ly=2.0):
    """Sinusoidal curvilinear grid of Eqs. 48-49 (reading of the garbled domain line: Lx = Ly = 2,
    dx = Lx/Nx, dy = Ly/Ny)."""
    dx, dy = Lx / N, Ly / N
    i = np.arange(N)[None, :]
    j = np.arange(N)[:, None]
    x = i * dx + A * np.sin(6.0 * math.pi * j * dy / Ly)
    y = j * dy + A * np.sin(6.0 * math.pi * i * dx / Lx)
    coords = np.zeros((3, 1, N, N))
    coords[0, 0] = x
    coords[1, 0] = y
    return coords


def euler_wave_exact(coords, t, u=1.0, v=-0.5):
    x, y = coords[0, 0], coords[1, 0]
    return 1.0 + 0.2 * np.sin(math.pi * (x + y - t * (u + v)))


def euler_wave(N=32, scheme=TENO5, dt=5e-4, A=0.04):
    """2D travelling density wave (Eq. 47) on the sinusoidal grid, periodic, inviscid, u = 1,
    v = -0.5, p = 1."""
    coords = euler_wave_grid(N, A)
    cfg = _base((N, N, 1), scheme=scheme, dt=dt, coords=coords, h=(2.0 / N, 2.0 / N, 1.0),
                L=(2.0, 2.0, 0.0))
    rho = euler_wave_exact(coords, 0.0)
    one = np.ones_like(rho)
    U = prim_to_cons(cfg["gamma"], rho, 1.0 * one, -0.5 * one, 0.0 * one, one)
    return cfg, U.reshape(5, 1, N, N)


def random_state(n, seed, gamma=1.4, Ma=1.0, amp=0.1, shocky=False):
    """Seeded smooth state (random low Fourier modes around a uniform flow) with optional
    embedded jumps; used by parity tests."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    Z, Y, X = np.meshgrid(np.arange(nz) / max(nz, 1), np.arange(ny) / max(ny, 1),
                          np.arange(nx) / max(nx, 1), indexing="ij")
    def field(base, a):
        f = np.full(X.shape, base)
        for _ in range(4):
            kx, ky, kz = rng.integers(1, 3, size=3)
            ph = rng.uniform(0, 2 * math.pi, size=3)
            f = f + a * rng.uniform(-1, 1) * np.sin(2 * math.pi * kx * X + ph[0]) * \
                np.sin(2 * math.pi * ky * Y + ph[1]) * np.sin(2 * math.pi * kz * Z + ph[2] + 0.3)
        return f
    rho = field(1.0, amp)
    u = field(0.3, amp)
    v = field(-0.2, amp) if ny > 1 else np.zeros_like(rho)
    w = field(0.1, amp) if nz > 1 else np.zeros_like(rho)
    p = field(1.0 / (gamma * Ma * Ma), amp / (gamma * Ma * Ma))
    if shocky:
        jump = (X > 0.5) ^ (Y > 0.37) if ny > 1 else (X > 0.5)
        rho = np.where(jump, rho * 0.35, rho)
        p = np.where(jump, p * 0.3, p)
    return prim_to_cons(gamma, rho, u, v, w, p)
