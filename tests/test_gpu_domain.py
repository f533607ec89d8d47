"""Split grids (osbli_domain_*): one grid in 2-4 z-slabs with halo exchanges between them gives
bitwise the state and residual of one handle on the whole grid -- FP64 and mixed precision,
characteristic and central schemes, inviscid and viscous (the second exchange, of the z viscous
fluxes), periodic and physical z faces, uneven slabs -- and is checked against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2007_14933_b300 import inputs as I
from paper_2007_14933_b300 import osbli

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14933_b300 import build
    build.build()
    osbli.load()


def closed_box(n=(20, 14, 23), viscous=True):
    """Uniform box with physical faces on every side: Dirichlet / zero-gradient in x, walls in y,
    zero-gradient / wall in z (T_wall = 1.2), a smooth state with a weak jump."""
    g, Ma, Tw = 1.4, 0.9, 1.2
    nx, ny, nz = n
    h = (0.2, 0.15, 0.1)
    z, y, x = np.meshgrid(np.arange(nz) * h[2], np.arange(ny) * h[1], np.arange(nx) * h[0], indexing="ij")
    T = Tw + 0.1 * np.sin(2 * y) + 0.05 * np.cos(3 * z)
    p = (1 + 0.05 * np.sin(x + z) + 0.2 * (x > 2.0)) / (g * Ma * Ma)
    rho = g * Ma * Ma * p / T
    u = 0.4 * np.sin(np.pi * y / (h[1] * (ny - 1))) * (1 + 0.1 * np.cos(z))
    w = 0.05 * np.sin(np.pi * y / (h[1] * (ny - 1))) * np.sin(3 * x)
    U = I.prim_to_cons(g, rho, u, 0.02 * np.sin(x) * np.sin(np.pi * y / (h[1] * (ny - 1))), w, p)
    for j in (0, -1):
        U[1:4, :, j, :] = 0.0
        U[4, :, j, :] = U[0, :, j, :] * Tw / (Ma * Ma * g * (g - 1))
    U[1:4, -1] = 0.0
    U[4, -1] = U[0, -1] * Tw / (Ma * Ma * g * (g - 1))
    face = np.zeros((5, nz, ny))
    face[0] = 1.1
    face[1] = 0.3
    face[4] = 1.0 / (g * Ma * Ma)
    cfg = dict(n=n, gamma=g, Re=400.0 if viscous else 0.0, Pr=0.72, Ma=Ma, dt=1e-3, scheme=I.TENO5,
               teno_ct=1e-5, bc=[[I.DIRICHLET, I.ZEROGRAD], [I.WALL, I.WALL], [I.ZEROGRAD, I.WALL]],
               h=h, T_wall=Tw, suth=110.4 / 288.0, bdata={(0, 0): face.reshape(5, -1)})
    return cfg, U


def _pair(cfg, U, nslab, precision, steps):
    s = osbli.Solver(cfg, precision=precision)
    s.set_state(U)
    R1 = s.residual()
    s.step(steps)
    U1 = s.get_state()
    s.close()
    d = osbli.Domain(cfg, nslab, precision=precision)
    d.set_state(U)
    R2 = d.residual()
    d.step(steps)
    U2 = d.get_state()
    nl, nc = d.launches_per_step()
    d.close()
    return R1, U1, R2, U2, nc


CASES = {
    "tgv_teno5_viscous": lambda: I.tgv(n=(24, 20, 26), Ma=1.25, scheme=I.TENO5),
    "tgv_central_viscous": lambda: I.tgv(n=(16, 18, 21), Ma=0.1, scheme=I.CENTRAL4),
    "tgv_weno_inviscid": lambda: I.tgv(n=(18, 16, 17), Ma=0.8, Re=0.0, scheme=I.WENO5JS),
    "closed_box_viscous": lambda: closed_box(),
    "closed_box_teno6_inviscid": lambda: (dict(closed_box(viscous=False)[0], scheme=I.TENO6),
                                          closed_box(viscous=False)[1]),
}


@pytest.mark.parametrize("nslab", [2, 3, 4])
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", [osbli.OSBLI_FP64, osbli.OSBLI_MIXED])
def test_split_is_bitwise_the_whole_grid(case, nslab, precision):
    cfg, U = CASES[case]()
    if precision == osbli.OSBLI_MIXED and cfg["scheme"] == I.CENTRAL4:
        pytest.skip("the mixed path is characteristic only")
    if cfg["bc"][2][0] != I.PERIODIC and cfg["n"][2] < 5 * nslab:
        pytest.skip("end slabs need 5 planes")
    R1, U1, R2, U2, copies = _pair(cfg, U, nslab, precision, steps=20)
    assert np.array_equal(R1, R2)
    assert np.array_equal(U1, U2)
    periodic = cfg["bc"][2][0] == I.PERIODIC
    faces = 2 * nslab if periodic else 2 * (nslab - 1)
    stages = 3
    assert copies == stages * faces * (2 if cfg.get("Re", 0.0) > 0 else 1)


def test_split_grid_matches_the_oracle():
    cfg, U = closed_box(n=(14, 12, 16))
    d = osbli.Domain(cfg, 3)
    d.set_state(U)
    d.step(10)
    Ug = d.get_state()
    d.close()
    o = O.Oracle(cfg)
    o.set_state(U)
    o.step(10)
    Uo = o.get_state()
    scale = np.abs(Uo).reshape(5, -1).max(axis=1)[:, None]
    assert (np.abs(Ug - Uo).reshape(5, -1) / scale).max() <= 1e-11


def test_split_reports_the_nonfinite_slab_and_rejects_short_slabs():
    cfg, U = I.tgv(n=(12, 10, 18), Ma=0.5, scheme=I.TENO5)
    U = U.copy()
    U[0, 15, 4, 5] = -1.0                    # negative density in the last of 3 slabs
    d = osbli.Domain(cfg, 3)
    d.set_state(U)
    with pytest.raises(osbli.OsbliError) as e:
        d.step(1)
    # within a step the NaNs reach the neighbouring slabs too (3 nodes per stage, periodic wrap)
    assert e.value.code == osbli.OSBLI_ENONFINITE and "slab" in str(e.value)
    d.close()
    with pytest.raises(osbli.OsbliError) as e:
        osbli.Domain(cfg, 7)                  # 18 planes in 7 slabs: 2-3 planes each
    assert e.value.code == osbli.OSBLI_EINVAL
    with pytest.raises(osbli.OsbliError):
        osbli.Domain(dict(cfg, sensor=1), 2, precision=osbli.OSBLI_MIXED)
