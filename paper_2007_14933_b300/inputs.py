"""Seeded / analytic problem set-ups shared by the CUDA path and the oracle.

This module holds problem descriptions, grids and initial states only: none of the method's
arithmetic (no flux, reconstruction, eigensystem, viscous term or time update).  A problem is a
plain dict:

    n        interior points (nx, ny, nz); 1 marks an inactive direction
    gamma, Re, Pr, Ma   (Re <= 0: inviscid)
    dt       fixed time step
    scheme   0 central 4th order, 1 WENO5-JS, 2 TENO5, 3 WENO-Z, 4 TENO6 (characteristic, Roe
             average)
    teno_ct  TENO cut-off C_T
    bc       bc[d][s]: 0 periodic, 1 zero-gradient, 2 isothermal wall, 3 Dirichlet, 4 inflow,
             5 adiabatic wall
    force    optional body force per unit volume (its work enters the energy equation)
    rk       0: 3-stage RK3 (default), 1: 5-stage RK4, 2: 3-stage SSP-RK3
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
    sbli()         shock / boundary-layer box [Sec. 6]: Mach 2, Re 1e4, similarity inflow,
                   isothermal wall, 10-degree oblique shock on the top boundary, tanh stretching
    laminar_channel() mixed isothermal / adiabatic-wall channel [Sec. 5.4] at its analytic state
    shu_osher()    Shu-Osher shock / density-wave interaction [Sec. 5.2]
    riemann2d(), riemann_ensemble()
                   four-quadrant 2D Riemann problems [Sec. 5.2] and seeded ensembles of them
"""
import math

import numpy as np

CENTRAL4, WENO5JS, TENO5, WENO5Z, TENO6 = 0, 1, 2, 3, 4
PERIODIC, ZEROGRAD, WALL, DIRICHLET, INFLOW, ADIABATIC = 0, 1, 2, 3, 4, 5


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


# ---------------------------------------------------------------------------------------------
# Shock / boundary-layer box (config of the learned-sensor workload): Mach 2 freestream over an
# isothermal wall, laminar similarity inflow, oblique shock imposed on the top boundary.
# ---------------------------------------------------------------------------------------------
def _rk4(fun, y0, t):
    y = np.zeros((len(t), len(y0)))
    y[0] = y0
    for i in range(len(t) - 1):
        h = t[i + 1] - t[i]
        k1 = fun(y[i])
        k2 = fun(y[i] + 0.5 * h * k1)
        k3 = fun(y[i] + 0.5 * h * k2)
        k4 = fun(y[i] + h * k3)
        y[i + 1] = y[i] + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return y


def similarity_profile(Ma=2.0, Pr=0.72, gamma=1.4, eta_max=12.0, npts=6001):
    """Compressible laminar boundary layer, Chapman-Rubesin constant C = 1, Howarth variable
    eta = Y / sqrt(2 nu x / U) (textbook similarity form): f''' + f f'' = 0 and
    T'' + Pr f T' + Pr (gamma-1) Ma^2 f''^2 = 0 with T'(0) = 0 (adiabatic wall), T(inf) = 1.
    Returns eta, f, f', T (T nondimensionalised by the freestream)."""
    eta = np.linspace(0.0, eta_max, npts)
    rhs = lambda v: np.array([v[1], v[2], -v[0] * v[2]])
    # scaling invariance of the Blasius equation: with F''(0) = 1 and F'(inf) = c,
    # f(eta) = c^(-1/2) F(c^(-1/2) eta) has f'(inf) = 1 and f''(0) = c^(-3/2)
    y1 = _rk4(rhs, np.array([0.0, 0.0, 1.0]), np.linspace(0.0, 2.0 * eta_max, npts))
    s = y1[-1, 1] ** -1.5
    y = _rk4(rhs, np.array([0.0, 0.0, s]), eta)
    f, fp, fpp = y[:, 0], y[:, 1], y[:, 2]
    # particular solution with T(0) = 0, T'(0) = 0; T = Tp + const satisfies T'(0) = 0
    c = Pr * (gamma - 1.0) * Ma * Ma
    z = np.zeros((npts, 2))
    for i in range(npts - 1):
        h = eta[i + 1] - eta[i]
        fi, fm, fe = f[i], 0.5 * (f[i] + f[i + 1]), f[i + 1]
        gi, gm, ge = fpp[i] ** 2, (0.5 * (fpp[i] + fpp[i + 1])) ** 2, fpp[i + 1] ** 2
        rhs = lambda v, ff, gg: np.array([v[1], -Pr * ff * v[1] - c * gg])
        k1 = rhs(z[i], fi, gi)
        k2 = rhs(z[i] + 0.5 * h * k1, fm, gm)
        k3 = rhs(z[i] + 0.5 * h * k2, fm, gm)
        k4 = rhs(z[i] + h * k3, fe, ge)
        z[i + 1] = z[i] + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    T = z[:, 0] + (1.0 - z[-1, 0])
    return eta, f, fp, T


def boundary_layer(y, Re, Ma=2.0, Pr=0.72, gamma=1.4):
    """u, v, T at wall distances y of the similarity layer scaled so that its displacement
    thickness is 1 (the length unit; Re = U delta* / nu)."""
    eta, f, fp, T = similarity_profile(Ma, Pr, gamma)
    d = np.diff(eta)
    I = np.sum(0.5 * ((T - fp)[1:] + (T - fp)[:-1]) * d)            # delta* = l I
    l = 1.0 / I
    G = np.concatenate([[0.0], np.cumsum(0.5 * (T[1:] + T[:-1]) * d)])
    ys = l * G
    u = np.interp(y, ys, fp, right=1.0)
    Ti = np.interp(y, ys, T, right=1.0)
    vv = -(T * f - fp * G) / (l * Re)                                 # v = T rho v
    v = np.interp(y, ys, vv, right=vv[-1])
    return u, v, Ti, T[0]


def oblique_shock(Ma, theta_deg, gamma=1.4):
    """Weak oblique shock for deflection theta (theta-beta-Ma relation) and the Rankine-Hugoniot
    post-shock state relative to a freestream rho = 1, |u| = 1, p = 1/(gamma Ma^2).  Returns
    beta (rad), rho2, p2, speed2 (the post-shock flow is turned by theta)."""
    th = np.radians(theta_deg)
    g = gamma

    def tan_theta(b):
        return 2.0 / np.tan(b) * (Ma ** 2 * np.sin(b) ** 2 - 1.0) / (Ma ** 2 * (g + np.cos(2 * b)) + 2.0)
    lo, hi = np.arcsin(1.0 / Ma) + 1e-9, np.radians(64.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if tan_theta(mid) < np.tan(th):
            lo = mid
        else:
            hi = mid
    b = 0.5 * (lo + hi)
    mn1 = Ma * np.sin(b)
    p21 = 1.0 + 2.0 * g / (g + 1.0) * (mn1 ** 2 - 1.0)
    r21 = (g + 1.0) * mn1 ** 2 / ((g - 1.0) * mn1 ** 2 + 2.0)
    mn2 = np.sqrt((1.0 + 0.5 * (g - 1.0) * mn1 ** 2) / (g * mn1 ** 2 - 0.5 * (g - 1.0)))
    M2 = mn2 / np.sin(b - th)
    T21 = p21 / r21
    speed2 = M2 / Ma * np.sqrt(T21)
    return b, r21, p21 / (g * Ma * Ma), speed2


def sbli(n=(512, 256, 64), Ma=2.0, Re=1e4, Pr=0.72, theta=10.0, stretch=3.0, L=(300.0, 60.0, 20.0),
         x_shock=20.0, scheme=TENO5, cfl=0.4, Tref=288.0):
    """Shock / boundary-layer box: uniform x in [0, Lx], wall-normal y_j = Ly (1 - tanh(s (1 -
    j/(Ny-1))) / tanh s), periodic z.  Isothermal wall at the similarity layer's adiabatic-wall
    temperature, inflow u, v, T from the similarity layer (pressure extrapolated), zero-gradient
    outlet, top Dirichlet: the inflow's outer state for x < x_shock, the Rankine-Hugoniot
    post-shock state of a theta-degree deflection of the freestream beyond.  Sutherland viscosity, T_s/T_ref = 110.4 / Tref."""
    g = 1.4
    nx, ny, nz = n
    Lx, Ly, Lz = L
    x = np.linspace(0.0, Lx, nx)
    j = np.arange(ny)
    y = Ly * (1.0 - np.tanh(stretch * (1.0 - j / (ny - 1))) / np.tanh(stretch))
    z = np.arange(nz) * Lz / nz if nz > 1 else np.zeros(1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    coords = np.stack([X, Y, Z])
    u1, v1, T1, Tw = boundary_layer(y, Re, Ma, Pr, g)
    p0 = 1.0 / (g * Ma * Ma)
    shape = (nz, ny, nx)
    u = np.broadcast_to(u1[None, :, None], shape).copy()
    v = np.broadcast_to(v1[None, :, None], shape).copy()
    T = np.broadcast_to(T1[None, :, None], shape).copy()
    p = np.full(shape, p0)
    rho = g * Ma * Ma * p / T
    U = prim_to_cons(g, rho, u, v, np.zeros(shape), p)
    U[1:4, :, 0, :] = 0.0
    U[4, :, 0, :] = U[0, :, 0, :] * Tw / (Ma * Ma * g * (g - 1.0))
    inflow = np.zeros((5, nz, ny))
    inflow[1] = u1[None, :]
    inflow[2] = v1[None, :]
    inflow[4] = T1[None, :]
    b, r2, p2, s2 = oblique_shock(Ma, theta, g)
    th = np.radians(theta)
    # top: the inflow's outer state upstream of x_shock (no spurious jump), the Rankine-Hugoniot
    # state of the turned freestream beyond
    top = np.zeros((5, nz, nx))
    after = (x >= x_shock)[None, :]
    top[0] = np.where(after, r2, 1.0 / T1[-1])
    top[1] = np.where(after, s2 * np.cos(th), u1[-1])
    top[2] = np.where(after, -s2 * np.sin(th), v1[-1])
    top[4] = np.where(after, p2, p0)
    cfg = _base(n, scheme=scheme, Re=Re, Pr=Pr, Ma=Ma, T_wall=Tw, suth=110.4 / Tref,
                bc=[[INFLOW, ZEROGRAD], [WALL, DIRICHLET], [PERIODIC, PERIODIC]],
                coords=coords, h=(1.0, 1.0, 1.0), L=(0.0, 0.0, Lz),
                bdata={(0, 0): inflow.reshape(5, -1), (1, 1): top.reshape(5, -1)})
    a = np.sqrt(g * p / rho)
    dx = Lx / (nx - 1)
    dy = np.diff(y).min()
    dz = Lz / nz if nz > 1 else np.inf
    cfg["dt"] = float(cfl / ((np.abs(u) + a).max() / dx + (np.abs(v) + a).max() / dy + a.max() / dz))
    cfg["beta_shock"] = float(np.degrees(b))
    return cfg, U


# ---------------------------------------------------------------------------------------------
# Four-quadrant 2D Riemann problems and seeded ensembles of them.
# ---------------------------------------------------------------------------------------------
ENSEMBLE_SIZES = (128, 192, 256, 384, 512, 768, 1024)


def riemann2d(N, quad, scheme=TENO5, cfl=0.4, gamma=1.4, ny=None):
    """Unit square, nodes at cell centres ((i + 1/2)/N), split at (1/2, 1/2); quad[q] = (rho, u, v,
    p) of quadrant q (0: x > 1/2, y > 1/2; 1: x < 1/2, y > 1/2; 2: x < 1/2, y < 1/2; 3: x > 1/2,
    y < 1/2), zero-gradient faces, inviscid, dt from the CFL number on the initial state."""
    nx = int(N)
    ny = int(ny or N)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    Y, X = np.meshgrid(y, x, indexing="ij")
    right, top = X > 0.5, Y > 0.5
    q = np.where(top, np.where(right, 0, 1), np.where(right, 3, 2))
    Q = np.asarray(quad, dtype=np.float64)
    rho, u, v, p = (Q[q, c] for c in range(4))
    U = prim_to_cons(gamma, rho, u, v, np.zeros_like(rho), p)[:, None]
    cfg = _base((nx, ny, 1), scheme=scheme, gamma=gamma, h=(1.0 / nx, 1.0 / ny, 1.0),
                bc=[[ZEROGRAD, ZEROGRAD], [ZEROGRAD, ZEROGRAD], [PERIODIC, PERIODIC]])
    cfg["dt"] = cfl_dt(cfg, U, cfl)
    return cfg, U


def riemann_ensemble(seed, nprob=64, sizes=ENSEMBLE_SIZES, scheme=TENO5, cfl=0.4):
    """Seeded ensemble: numpy's PCG64 generator seeded with `seed` draws, per problem, N uniformly
    from `sizes` and then four quadrant states with rho, p ~ U[0.1, 1.5] and u, v ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nprob):
        N = int(rng.choice(sizes))
        quad = np.empty((4, 4))
        for k in range(4):
            quad[k, 0] = rng.uniform(0.1, 1.5)
            quad[k, 1] = rng.uniform(-1.0, 1.0)
            quad[k, 2] = rng.uniform(-1.0, 1.0)
            quad[k, 3] = rng.uniform(0.1, 1.5)
        out.append(riemann2d(N, quad, scheme=scheme, cfl=cfl))
    return out


def shu_osher(N=320, scheme=WENO5Z, dt=2e-4):
    """Shu-Osher shock / density-wave interaction [Sec. 5.2]: x in [-5, 5], nodes at cell centres,
    (rho, u, p) = (3.857143, 2.629369, 10.33333) for x < -4, else (1 + 0.2 sin 5x, 0, 1) (the
    printed right state lists u and p as (1.0, 0.0); the textbook problem has u = 0, p = 1),
    Dirichlet faces holding the initial end states, dt = 2e-4 (t = 1.8 after 9000 steps)."""
    x = -5.0 + (np.arange(N) + 0.5) * 10.0 / N
    left = x < -4.0
    rho = np.where(left, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
    u = np.where(left, 2.629369, 0.0)
    p = np.where(left, 10.33333, 1.0)
    z = np.zeros(N)
    cfg = _base((N, 1, 1), scheme=scheme, dt=dt, h=(10.0 / N, 1.0, 1.0),
                bc=[[DIRICHLET, DIRICHLET], [PERIODIC, PERIODIC], [PERIODIC, PERIODIC]])
    lo = np.array([3.857143, 2.629369, 0.0, 0.0, 10.33333]).reshape(5, 1)
    hi = np.array([1.0 + 0.2 * np.sin(5.0 * 5.0), 0.0, 0.0, 0.0, 1.0]).reshape(5, 1)
    cfg["bdata"] = {(0, 0): lo, (0, 1): hi}
    U = prim_to_cons(cfg["gamma"], rho, u, z, z, p).reshape(5, 1, 1, N)
    return cfg, U, x


def laminar_channel_exact(y, Re=90.0, Pr=0.72, Ma=0.01, gamma=1.4):
    """Analytic laminar channel [Sec. 5.4]: isothermal wall (T = 1) at y = -1, adiabatic wall at
    y = 1, constant viscosity: u = Re (1 - y^2) / 2, T = 1 - Re^2 Ma^2 Pr (gamma-1) (y^4 - 4y - 5)/12."""
    u = Re * (1.0 - y ** 2) / 2.0
    T = 1.0 - Re ** 2 * Ma ** 2 * Pr * (gamma - 1.0) * (y ** 4 - 4.0 * y - 5.0) / 12.0
    return u, T


def laminar_channel(Nx=32, Ny=64, Re=90.0, Pr=0.72, Ma=0.01, scheme=CENTRAL4, dt=1e-4):
    """The channel of Sec. 5.4 on Lx = 2 pi (periodic), y in [-1, 1] with wall nodes at both ends,
    at its analytic steady state: unit body force along x (its work u in the energy equation),
    uniform pressure 1/(gamma Ma^2), rho = 1/T, constant viscosity."""
    g = 1.4
    x = np.arange(Nx) * 2.0 * np.pi / Nx
    y = np.linspace(-1.0, 1.0, Ny)
    u1, T1 = laminar_channel_exact(y, Re, Pr, Ma, g)
    shape = (1, Ny, Nx)
    u = np.broadcast_to(u1[None, :, None], shape)
    T = np.broadcast_to(T1[None, :, None], shape)
    p = np.full(shape, 1.0 / (g * Ma * Ma))
    rho = 1.0 / T
    z = np.zeros(shape)
    U = prim_to_cons(g, rho, u, z, z, p)
    cfg = _base((Nx, Ny, 1), scheme=scheme, Re=Re, Pr=Pr, Ma=Ma, dt=dt, T_wall=1.0,
                h=(2.0 * np.pi / Nx, 2.0 / (Ny - 1), 1.0),
                bc=[[PERIODIC, PERIODIC], [WALL, ADIABATIC], [PERIODIC, PERIODIC]])
    cfg["force"] = (1.0, 0.0, 0.0)
    return cfg, U, y
