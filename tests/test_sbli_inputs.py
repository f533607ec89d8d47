"""Pins of the shock / boundary-layer set-up (no GPU): the similarity inflow and the oblique-shock
state imposed on the top boundary, against textbook values and conservation across the shock."""
import numpy as np
import pytest

from paper_2007_14933_b300 import inputs as I


def test_blasius_wall_shear():
    # f''' + f f'' = 0, f(0) = f'(0) = 0, f'(inf) = 1: f''(0) = 0.469600 (Howarth's value)
    eta, f, fp, T = I.similarity_profile(Ma=0.0)
    h = eta[1] - eta[0]
    fpp0 = (-3 * fp[0] + 4 * fp[1] - fp[2]) / (2 * h)
    assert abs(fpp0 - 0.469600) < 2e-5
    assert abs(fp[-1] - 1.0) < 1e-6
    assert np.allclose(T, 1.0)          # Ma = 0: no heating


def test_crocco_busemann_at_unit_prandtl():
    # Pr = 1, adiabatic wall: T = 1 + (gamma-1)/2 Ma^2 (1 - f'^2) exactly (total enthalpy constant)
    Ma, g = 2.0, 1.4
    eta, f, fp, T = I.similarity_profile(Ma=Ma, Pr=1.0, gamma=g)
    np.testing.assert_allclose(T, 1.0 + 0.5 * (g - 1) * Ma ** 2 * (1 - fp ** 2), atol=2e-6)


def test_recovery_factor_near_sqrt_prandtl():
    # laminar recovery factor r = (T_aw - 1) / ((gamma-1)/2 Ma^2) ~ Pr^(1/2) for air
    Ma, g, Pr = 2.0, 1.4, 0.72
    _, _, _, T = I.similarity_profile(Ma=Ma, Pr=Pr, gamma=g)
    r = (T[0] - 1.0) / (0.5 * (g - 1) * Ma ** 2)
    assert abs(r - np.sqrt(Pr)) < 0.01


def test_displacement_thickness_is_the_length_unit():
    cfg, U = I.sbli(n=(8, 400, 1), L=(10.0, 40.0, 1.0), stretch=2.0)
    y = cfg["coords"][1, 0, :, 0]
    rho, u = U[0, 0, :, 0], U[1, 0, :, 0] / U[0, 0, :, 0]
    dstar = np.sum(0.5 * ((1 - rho * u)[1:] + (1 - rho * u)[:-1]) * np.diff(y))
    assert abs(dstar - 1.0) < 2e-3
    # wall node: no slip at the wall temperature, freestream at the top
    assert U[1, 0, 0, 0] == 0.0 and U[2, 0, 0, 0] == 0.0
    assert abs(u[-1] - 1.0) < 1e-6 and abs(rho[-1] - 1.0) < 1e-6


def test_oblique_shock_mach2_deflection10():
    # theta-beta-Ma tables (e.g. NACA 1135): Ma 2, theta 10 deg -> beta 39.31 deg,
    # p2/p1 = 1.7066, rho2/rho1 = 1.4584, Ma2 = 1.6405
    g, Ma = 1.4, 2.0
    b, r2, p2, s2 = I.oblique_shock(Ma, 10.0, g)
    p1 = 1.0 / (g * Ma * Ma)
    assert abs(np.degrees(b) - 39.314) < 2e-3
    assert abs(p2 / p1 - 1.7066) < 2e-4
    assert abs(r2 - 1.4584) < 2e-4
    M2 = s2 / np.sqrt(g * p2 / r2)
    assert abs(M2 - 1.6405) < 2e-4


@pytest.mark.parametrize("Ma,theta", [(2.0, 10.0), (3.0, 15.0), (1.6, 5.0)])
def test_oblique_shock_conserves_mass_momentum_energy(Ma, theta):
    """Across the shock (normal n at beta to the freestream): rho u_n, rho u_n^2 + p and
    h + q^2/2 are continuous, tangential velocity unchanged, flow turned by theta."""
    g = 1.4
    b, r2, p2, s2 = I.oblique_shock(Ma, theta, g)
    th = np.radians(theta)
    p1 = 1.0 / (g * Ma * Ma)
    # the shock descends from the top boundary: tangent (cos b, -sin b), normal pointing downstream
    t = np.array([np.cos(b), -np.sin(b)])
    n = np.array([np.sin(b), np.cos(b)])
    u1 = np.array([1.0, 0.0])
    u2 = s2 * np.array([np.cos(th), -np.sin(th)])
    assert abs(u1 @ t - u2 @ t) < 1e-12
    un1, un2 = u1 @ n, u2 @ n
    assert un1 > 0 and un2 > 0
    assert abs(un1 - r2 * un2) < 1e-12
    assert abs((un1 ** 2 + p1) - (r2 * un2 ** 2 + p2)) < 1e-12
    h1 = g / (g - 1) * p1 + 0.5
    h2 = g / (g - 1) * p2 / r2 + 0.5 * s2 ** 2
    assert abs(h1 - h2) < 1e-12
    assert p2 > p1                                 # compression (entropy increases)
