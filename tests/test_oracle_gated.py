"""Pins of the oracle's gated convective form (no GPU).

The gated form is the learned-sensor extension: a cell gate chooses, per interface, the
characteristic WENO/TENO flux of Sec. 2.2 (either adjacent cell gated, or a strong jump in the
six-node stencil) or the central 4th-order interface flux [7(F_i + F_{i+1}) - (F_{i-1} +
F_{i+2})]/12 (Sec. 2.6, Eq. 28 in flux form with the sign of the Sec. 4 kernel).  These tests tie
it to the oracle's separately pinned central (ORC_CENTRAL4, exact on quartics, closed-form
viscous residuals) and TENO5 paths, and to invariants a plausible slip (a gate index off by one,
a strong-jump window of the wrong width, a decision taken per point instead of per interface)
would break.
"""
import numpy as np

import oracle as O
from paper_2007_14933_b300 import inputs as I


def _res(cfg, U, gate=None, jump=1.5, **kw):
    o = O.Oracle(dict(cfg, **kw))
    o.set_state(U)
    if gate is not None:
        o.set_gate(gate, jump)
    return o.residual()


def _rel(a, b):
    sc = np.abs(b).reshape(5, -1).max(axis=1)[:, None]
    sc[sc == 0] = 1.0
    return float((np.abs(a - b).reshape(5, -1) / sc).max())


def line_state(n, seed, jump_at=None, ratio=2.0):
    """1D periodic line of smooth low-amplitude data, optionally with one density/pressure jump of
    the given ratio between nodes jump_at and jump_at + 1."""
    rng = np.random.default_rng(seed)
    x = np.arange(n) / n
    rho = 1.0 + 0.05 * np.sin(2 * np.pi * x + rng.uniform(0, 6))
    u = 0.3 + 0.05 * np.cos(2 * np.pi * x + rng.uniform(0, 6))
    p = 0.7 + 0.03 * np.sin(4 * np.pi * x + rng.uniform(0, 6))
    if jump_at is not None:
        hi = np.arange(n) > jump_at
        rho = np.where(hi, rho / ratio, rho)
        p = np.where(hi, p / ratio, p)
    z = np.zeros(n)
    return I.prim_to_cons(1.4, rho, u, z, z, p).reshape(5, 1, 1, n)


def _sc(R):
    """Per-variable scale of a line residual [5][n] (1 for the identically zero v, w rows)."""
    sc = np.abs(R).max(axis=1)
    sc[sc == 0] = 1.0
    return sc


def line_cfg(n, bc=0):
    return dict(n=(n, 1, 1), gamma=1.4, Re=0.0, Ma=1.0, scheme=I.TENO5, teno_ct=1e-5,
                bc=[[bc, bc], [0, 0], [0, 0]], h=(1.0 / n, 1.0, 1.0))


def test_zero_gate_on_smooth_periodic_flow_is_the_central_scheme():
    """No gated cell and no strong jump: every interface takes the central interface flux, whose
    differences telescope to the 4th-order central derivative of the CENTRAL4 path (inviscid and
    viscous, 3D TGV and a seeded random smooth field)."""
    cases = [I.tgv(n=(12, 10, 8), Ma=0.4, Re=0.0, scheme=I.TENO5),
             I.tgv(n=(12, 10, 8), Ma=0.4, Re=200.0, scheme=I.TENO5)]
    n = (11, 9, 7)
    cases.append((dict(n=n, gamma=1.4, Re=0.0, Ma=1.0, scheme=I.WENO5JS, bc=[[0, 0]] * 3,
                       h=(0.1, 0.2, 0.3)), I.random_state(n, seed=4)))
    for cfg, U in cases:
        gate = np.zeros(U.shape[1:], np.uint8)
        Rg = _res(cfg, U, gate)
        Rc = _res(cfg, U, scheme=I.CENTRAL4)
        assert _rel(Rg, Rc) <= 1e-13


def test_every_cell_gated_is_the_characteristic_scheme():
    """All cells gated: every interface is characteristic, so the residual is the plain TENO5
    (or WENO5-JS) one, to the bit, on smooth and on discontinuous data."""
    n = (13, 9, 7)
    for scheme in (I.TENO5, I.WENO5JS):
        for shocky in (False, True):
            U = I.random_state(n, seed=3, shocky=shocky)
            cfg = dict(n=n, gamma=1.4, Re=0.0, Ma=1.0, scheme=scheme, bc=[[0, 0]] * 3,
                       h=(0.1, 0.2, 0.3))
            Rg = _res(cfg, U, np.ones(U.shape[1:], np.uint8))
            Rp = _res(cfg, U)
            assert np.array_equal(Rg, Rp)


def test_one_gated_cell_changes_only_its_own_interfaces():
    """Cell 7 of a periodic line gated: its two interfaces 6.5 and 7.5 are characteristic, every
    other one central.  So R equals the central residual away from nodes 6..8, equals the TENO5
    residual at node 7, and over nodes 6..8 it sums to the central sum (the outer interfaces 5.5
    and 8.5 are central on both)."""
    n = 24
    cfg, U = line_cfg(n), line_state(n, seed=1)
    gate = np.zeros((1, 1, n), np.uint8)
    gate[0, 0, 7] = 1
    Rg = _res(cfg, U, gate)[:, 0, 0, :]
    Rc = _res(cfg, U, scheme=I.CENTRAL4)[:, 0, 0, :]
    Rt = _res(cfg, U)[:, 0, 0, :]
    sc = _sc(Rc)[:, None]
    away = [i for i in range(n) if abs(i - 7) >= 2]
    assert (np.abs(Rg[:, away] - Rc[:, away]) / sc).max() <= 1e-12
    assert (np.abs(Rg[:, 7] - Rt[:, 7]) / sc[:, 0]).max() <= 1e-12
    assert (np.abs(Rg[:, 6] - Rc[:, 6]) / sc[:, 0]).max() > 1e-8        # the gate did act
    assert (np.abs(Rg[:, 6:9].sum(axis=1) - Rc[:, 6:9].sum(axis=1)) / sc[:, 0]).max() <= 1e-12


def test_strong_jump_makes_its_six_node_window_characteristic():
    """A density / pressure jump of ratio 2 between nodes 12 and 13, nothing gated: the interfaces
    m + 1/2 whose stencil m-2..m+3 holds the pair (12, 13) -- m = 10..14 -- are characteristic.
    So nodes 11..14 (both interfaces characteristic) carry the TENO5 residual, and nodes <= 9 or
    >= 16 (both interfaces central) the central one."""
    n = 28
    cfg, U = line_cfg(n), line_state(n, seed=2, jump_at=12, ratio=2.0)
    # a periodic line also jumps back at the seam (node n-1 -> node 0)
    gate = np.zeros((1, 1, n), np.uint8)
    Rg = _res(cfg, U, gate)[:, 0, 0, :]
    Rc = _res(cfg, U, scheme=I.CENTRAL4)[:, 0, 0, :]
    Rt = _res(cfg, U)[:, 0, 0, :]
    sc = _sc(Rt)[:, None]
    for i in range(11, 15):
        assert (np.abs(Rg[:, i] - Rt[:, i]) / sc[:, 0]).max() <= 1e-12, i
    # the seam jump's window is m = n-3..n+1 (mod n): nodes n-2..n+1 characteristic
    central = [i for i in range(n) if (i <= 9 and i >= 3) or (16 <= i <= n - 5)]
    assert (np.abs(Rg[:, central] - Rc[:, central]) / sc).max() <= 1e-12
    for i in (10, 15):    # one interface of each kind: neither pure form
        assert (np.abs(Rg[:, i] - Rt[:, i]) / sc[:, 0]).max() > 1e-8
        assert (np.abs(Rg[:, i] - Rc[:, i]) / sc[:, 0]).max() > 1e-8
    # a ratio just below the threshold leaves the window central
    U2 = line_state(n, seed=2, jump_at=12, ratio=1.4)
    Rg2 = _res(cfg, U2, gate)[:, 0, 0, :]
    Rc2 = _res(cfg, U2, scheme=I.CENTRAL4)[:, 0, 0, :]
    assert _rel(Rg2.reshape(5, 1, 1, n), Rc2.reshape(5, 1, 1, n)) <= 1e-13


def test_ghost_nodes_take_the_gate_of_the_nearest_interior_node():
    """Zero-gradient line with only cell 0 gated: its interfaces -1/2 (ghost -1 takes cell 0's
    gate) and 1/2 are characteristic, so node 0 carries the TENO5 residual; cell n-1 is not
    gated, so node n-1 keeps the central interface fluxes of the ghosted data."""
    n = 20
    cfg, U = line_cfg(n, bc=I.ZEROGRAD), line_state(n, seed=5)
    gate = np.zeros((1, 1, n), np.uint8)
    gate[0, 0, 0] = 1
    Rg = _res(cfg, U, gate)[:, 0, 0, :]
    Rt = _res(cfg, U)[:, 0, 0, :]
    sc = _sc(Rt)
    assert (np.abs(Rg[:, 0] - Rt[:, 0]) / sc).max() <= 1e-12
    assert (np.abs(Rg[:, n - 1] - Rt[:, n - 1]) / sc).max() > 1e-8
    # node n-1 by hand: central fluxes at n-3/2 and n-1/2 from the zero-gradient ghosts
    g = 1.4
    Ue = np.concatenate([U[:, 0, 0, :], np.repeat(U[:, 0, 0, -1:], 3, axis=1)], axis=1)
    rho, m, E = Ue[0], Ue[1], Ue[4]
    u = m / rho
    p = (g - 1) * (E - 0.5 * rho * u * u)
    F = np.stack([m, m * u + p, 0 * m, 0 * m, (E + p) * u])

    def fc(i):
        return (7 * (F[:, i] + F[:, i + 1]) - (F[:, i - 1] + F[:, i + 2])) / 12
    R_hand = -(fc(n - 1) - fc(n - 2)) * n
    assert (np.abs(Rg[:, n - 1] - R_hand) / sc).max() <= 1e-12


def test_gated_form_conserves_on_periodic_grids():
    """Whatever the gate, each interface flux enters its two nodes with opposite signs, so the
    residual sums to zero over a periodic box (a decision taken per node instead of per interface
    would break this)."""
    n = (12, 10, 8)
    rng = np.random.default_rng(7)
    U = I.random_state(n, seed=6, shocky=True)
    cfg = dict(n=n, gamma=1.4, Re=0.0, Ma=1.0, scheme=I.TENO5, bc=[[0, 0]] * 3, h=(0.1, 0.1, 0.1))
    gate = (rng.random(U.shape[1:]) < 0.35).astype(np.uint8)
    R = _res(cfg, U, gate)
    tot = R.reshape(5, -1).sum(axis=1)
    sc = np.abs(R).reshape(5, -1).sum(axis=1)
    assert (np.abs(tot) / sc).max() <= 1e-13
