"""Pins of the sensor reference (oracle/sensor.py) and of the oracle's TENO cut-off labels."""
import numpy as np

import oracle as O
from oracle import sensor as S
from paper_2007_14933_b300 import inputs as I


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = S.init_weights(1).astype(np.float64) + rng.normal(0, 0.05, S.NPARAM)
    X = rng.normal(0, 0.5, (40, S.NF))
    y = (rng.uniform(size=40) < 0.3).astype(np.float64)
    L, g = S.loss_and_grad(w, X, y, pos_weight=3.0)
    idx = rng.choice(S.NPARAM, 60, replace=False)
    for i in idx:
        e = np.zeros(S.NPARAM)
        e[i] = 1e-6
        Lp, _ = S.loss_and_grad(w + e, X, y, 3.0)
        Lm, _ = S.loss_and_grad(w - e, X, y, 3.0)
        fd = (Lp - Lm) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_forward_matches_loss_probabilities():
    rng = np.random.default_rng(2)
    w = S.init_weights(3).astype(np.float64)
    X = rng.normal(size=(8, S.NF))
    z, p = S.forward(w, X)
    assert np.all((p > 0) & (p < 1))
    np.testing.assert_allclose(p, 1 / (1 + np.exp(-z)))


def _ghosted(cfg, U):
    o = O.Oracle(cfg)
    o.set_state(U)
    return o.ghosted()


def test_features_vanish_on_uniform_flow_and_are_galilean():
    cfg, U = I.tgv(8, Ma=0.5)
    g = cfg["gamma"]
    one = np.ones((8, 8, 8))
    Uu = I.prim_to_cons(g, 1.3 * one, 0.2 * one, -0.1 * one, 0.05 * one, 0.9 * one)
    F = S.features(_ghosted(cfg, Uu), cfg["n"], g)
    assert np.abs(F).max() < 1e-14
    rho = U[0]
    u = U[1:4] / rho
    p = (g - 1) * (U[4] - 0.5 * rho * (u ** 2).sum(0))
    F1 = S.features(_ghosted(cfg, U), cfg["n"], g)
    U2 = I.prim_to_cons(g, 2 * rho, u[0] + 0.3, u[1] - 0.2, u[2] + 0.1, 2 * p)   # shift u, scale rho,p
    F2 = S.features(_ghosted(cfg, U2), cfg["n"], g)
    # velocity features scale with 1/a (a unchanged when rho and p scale together): equal
    np.testing.assert_allclose(F1, F2, atol=1e-12)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -3.14159], dtype=np.float32)
    r = S.bf16_round(x)
    np.testing.assert_array_equal(r[:3], [1.0, 1.0, 1.0 + 4 * 2 ** -9])   # ties to even
    assert abs(r[3] + 3.140625) < 1e-7


def test_teno_labels_mark_sod_waves_only():
    cfg, U, x = I.sod(scheme=I.TENO5)
    o = O.Oracle(cfg)
    o.set_state(U)
    o.step(400)                    # t = 0.1
    lab = o.labels()[0, 0]
    shock = np.argmin(np.abs(x - (0.5 + 1.7522 * 0.1)))
    assert lab[shock - 3:shock + 4].any()
    assert not lab[:100].any() and not lab[320:].any()      # undisturbed states
