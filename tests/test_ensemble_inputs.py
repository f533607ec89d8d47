"""Ensemble set-up (no GPU): seeded sizes and states, quadrant layout, CFL time step, and the
C ABI's validation of ensemble members (rejected before any device work)."""
import ctypes

import numpy as np
import pytest

from paper_2007_14933_b300 import inputs as I


def test_riemann_ensemble_is_seeded_and_in_range():
    a = I.riemann_ensemble(3, nprob=16)
    b = I.riemann_ensemble(3, nprob=16)
    c = I.riemann_ensemble(4, nprob=16)
    assert [x[0]["n"] for x in a] == [x[0]["n"] for x in b]
    assert all(np.array_equal(x[1], y[1]) for x, y in zip(a, b))
    assert [x[0]["n"] for x in a] != [x[0]["n"] for x in c] or \
        not all(np.array_equal(x[1], y[1]) for x, y in zip(a, c))
    for cfg, U in a:
        assert cfg["n"][0] in I.ENSEMBLE_SIZES and cfg["n"][0] == cfg["n"][1] and cfg["n"][2] == 1
        rho = U[0]
        u = U[1] / rho
        p = 0.4 * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
        assert rho.min() >= 0.1 and rho.max() <= 1.5
        assert p.min() >= 0.1 - 1e-12 and p.max() <= 1.5 + 1e-12
        assert np.abs(u).max() <= 1.0


def test_quadrant_layout_and_cfl():
    quad = [(1.0, 0.1, 0.2, 1.0), (0.5, 0.0, 0.0, 0.4), (0.2, -0.3, 0.0, 0.3), (0.8, 0.0, 0.5, 0.9)]
    cfg, U = I.riemann2d(8, quad, cfl=0.4)
    rho = U[0, 0]
    assert rho[7, 7] == 1.0 and rho[7, 0] == 0.5 and rho[0, 0] == 0.2 and rho[0, 7] == 0.8
    assert rho[3, 3] == 0.2 and rho[4, 4] == 1.0      # split between nodes 3 and 4 (x = 1/2)
    # dt = CFL / max(sum_d (|u_d| + a) / h_d), h = 1/8
    g = 1.4
    s = max((abs(u) + np.sqrt(g * p / r)) * 8 + (abs(v) + np.sqrt(g * p / r)) * 8 for r, u, v, p in quad)
    assert abs(cfg["dt"] - 0.4 / s) <= 1e-15 * cfg["dt"]


def test_ensemble_create_validates_members_without_a_device():
    from paper_2007_14933_b300 import osbli
    try:
        osbli.load()
    except OSError:
        pytest.skip("library not built")
    cfg, _ = I.riemann2d(16, [(1, 0, 0, 1)] * 4)
    good = osbli.make_params(cfg, osbli.OSBLI_MIXED)
    bad_visc = osbli.make_params(dict(cfg, Re=100.0), osbli.OSBLI_MIXED)
    bad_wall = osbli.make_params(dict(cfg, bc=[[I.WALL, I.ZEROGRAD], [I.ZEROGRAD, I.ZEROGRAD], [0, 0]]),
                                 osbli.OSBLI_MIXED)
    bad_prec = osbli.make_params(cfg, osbli.OSBLI_FP64)
    for params, word in (([good, bad_visc], "inviscid"), ([good, bad_wall], "PERIODIC or ZEROGRAD"),
                         ([good, bad_prec], "precision")):
        with pytest.raises(osbli.OsbliError) as e:
            osbli.osbli_ensemble_create(params)
        assert e.value.code == osbli.OSBLI_EINVAL and "member 1" in str(e.value) and word in str(e.value)
