"""Shock / boundary-layer box (tanh-stretched rectilinear grid, isothermal wall, similarity
inflow, oblique shock on the top boundary, Sutherland viscosity) through the C ABI against the
oracle, on a reduced box.

Rectilinear grids run the Cartesian kernels with per-line factors S_dd / Jinv; the oracle runs
its general curvilinear form.  Bars: plain FP64 as for every FP64 parity test (1e-11 of each
variable's maximum, ambiguous TENO cut-offs bounded separately); mixed precision relative L2
<= 1e-5 after the steps; the learned gate accepts the rectilinear grid and refuses a general one.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_14933_b300 import inputs as I
from paper_2007_14933_b300 import osbli
from tests.test_gpu_parity import check_residual, relerr, run_pair
from tests.test_gpu_mixed import l2rel, mixed_vs_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14933_b300 import build
    build.build()
    osbli.load()


def small_sbli(scheme=I.TENO5, n=(45, 38, 6)):
    return I.sbli(n=n, L=(45.0, 15.0, 3.0), x_shock=12.0, scheme=scheme)


@pytest.mark.parametrize("scheme", [I.TENO5, I.WENO5JS])
def test_sbli_residual_fp64(scheme):
    cfg, U = small_sbli(scheme)
    check_residual(cfg, U)


def test_sbli_steps_fp64():
    cfg, U = small_sbli()
    Ug, Uo = run_pair(cfg, U, 15)
    assert relerr(Ug, Uo) <= 1e-11


def test_sbli_mixed_runs_the_delta_path_and_matches():
    cfg, U = small_sbli()
    s = osbli.Solver(cfg, precision=osbli.OSBLI_MIXED)
    s.set_state(U)
    names = [nm for nm, _ in s.profile_residual()]
    assert "patch" in names            # Cartesian delta kernels (with the FP64 fix pass) ran
    s.close()
    Ug, Uo = mixed_vs_oracle(cfg, U, 15)
    assert l2rel(Ug, Uo) <= 1e-5


def test_sbli_labels_match_oracle():
    cfg, U = small_sbli()
    s = osbli.Solver(cfg)
    s.set_state(U)
    s.step(10)
    U = s.get_state()
    lg = s.labels()
    o = O.Oracle(cfg)
    o.set_state(U)
    lo = o.labels()
    assert lo.any()
    assert (lg != lo).mean() <= 0.002


def test_sbli_learned_gate_accepted_on_rectilinear_grid():
    from paper_2007_14933_b300 import sensor as SN
    cfg, U = small_sbli()
    s = osbli.Solver(dict(cfg, sensor=1), precision=osbli.OSBLI_MIXED)
    s.set_state(U)
    s.set_sensor(SN.default_weights(3), 0.5)
    s.step(5)
    Ug = s.get_state()
    d = s.diagnostics()
    assert np.isfinite(Ug).all()
    assert 0.0 <= d[9] <= 1.0


def test_sbli_gate_on_every_cell_is_the_mixed_path():
    """Rectilinear box with inflow / outflow in x and wall / Dirichlet top in y: with every cell
    flagged the gated passes (x and y fused, then z) record every interface and the patch pass
    recomputes each, so 5 steps match the ungated mixed path to FP32 rounding order."""
    from paper_2007_14933_b300 import sensor as SN
    cfg, U = small_sbli()
    m = osbli.Solver(cfg, precision=osbli.OSBLI_MIXED)
    m.set_state(U)
    m.step(5)
    Um = m.get_state()
    m.close()
    g = osbli.Solver(dict(cfg, sensor=1), precision=osbli.OSBLI_MIXED)
    g.set_state(U)
    g.set_sensor(SN.default_weights(3), 1e-9)
    g.step(5)
    Ug = g.get_state()
    assert g.diagnostics()[9] > 0.99
    g.close()
    a, b = Ug.reshape(5, -1), Um.reshape(5, -1)
    nb = [np.linalg.norm(b[v]) for v in range(5)]
    nb[1] = nb[2] = nb[3] = max(nb[1:4])
    assert max(np.linalg.norm(a[v] - b[v]) / nb[v] for v in range(5)) <= 1e-6


def test_learned_gate_refuses_general_curvilinear_grid():
    cfg, U = I.euler_wave(24, scheme=I.TENO5)
    with pytest.raises(osbli.OsbliError) as e:
        osbli.Solver(dict(cfg, sensor=1), precision=osbli.OSBLI_MIXED)
    assert e.value.code == osbli.OSBLI_EINVAL
