"""Shu-Osher shock / density-wave interaction (Sec. 5.2) with WENO-Z and WENO-JS.

Parity: the FP64 GPU path against the oracle after 1800 steps (t = 0.36), bar 1e-11 as every FP64
parity test.  Accuracy: at t = 1.8 on N = 320, the density against an N = 3200 solution of the
same scheme (cell averages of the fine solution over each coarse cell): WENO-Z is the less
dissipative of the two (the paper's motivation for WENO-Z, Sec. 2.4), and the shock sits within
one coarse cell of the fine solution's.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_14933_b300 import inputs as I
from paper_2007_14933_b300 import osbli
from tests.test_gpu_parity import relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14933_b300 import build
    build.build()
    osbli.load()


def run(N, scheme, steps):
    cfg, U, x = I.shu_osher(N, scheme=scheme)
    s = osbli.Solver(cfg)
    s.set_state(U)
    s.step(steps)
    V = s.get_state()
    s.close()
    return cfg, U, x, V


def test_shu_osher_wenoz_matches_oracle():
    cfg, U, x, V = run(320, I.WENO5Z, 1800)
    o = O.Oracle(cfg)
    o.set_state(U)
    o.step(1800)
    assert relerr(V, o.get_state()) <= 1e-11


def _shock(x, rho):
    # the main shock: the rightmost place where density falls below the pre-shock wave's maximum
    i = np.where((rho[:-1] > 1.5) & (rho[1:] <= 1.5))[0][-1]
    return x[i]


def test_shu_osher_wenoz_less_dissipative_than_wenojs():
    err = {}
    for scheme in (I.WENO5Z, I.WENO5JS):
        _, _, xc, Vc = run(320, scheme, 9000)
        _, _, xf, Vf = run(3200, scheme, 9000)
        rc = Vc[0, 0, 0]
        rf = Vf[0, 0, 0].reshape(320, 10).mean(axis=1)
        err[scheme] = np.abs(rc - rf).mean()
        assert abs(_shock(xc, rc) - _shock(xc, rf)) <= 10.0 / 320 + 1e-12
    print("Shu-Osher N=320 L1(rho) vs N=3200: WENO-Z %.4f, WENO-JS %.4f" % (err[I.WENO5Z], err[I.WENO5JS]))
    assert err[I.WENO5Z] < err[I.WENO5JS]
