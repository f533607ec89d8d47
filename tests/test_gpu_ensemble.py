"""Ensembles of independent 2D Riemann problems through the C ABI.

Bars: plain FP64 members against the oracle as every FP64 parity test (1e-11 of each variable's
maximum, momentum components sharing one scale) and bitwise equal to the same problem run on its
own handle; mixed members within 1e-7 of their own handle after one step (the same FP32
expressions compiled into different kernels: fused multiply-add choices may differ by an FP32
rounding, which TENO cut-offs at discontinuities can amplify over many steps) and within the
mixed path's bars of the oracle; chunk choice and autotuning bitwise neutral (same kernels); the
launch count of a step independent of the member count.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_14933_b300 import inputs as I
from paper_2007_14933_b300 import osbli
from tests.test_gpu_parity import relerr
from tests.test_gpu_mixed import l2rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14933_b300 import build
    build.build()
    osbli.load()


def small_members(scheme=I.TENO5, seed=7):
    rng = np.random.default_rng(seed)
    shapes = [(24, 24), (32, 20), (40, 36), (17, 29), (48, 48), (300, 9)]
    out = []
    for nx, ny in shapes:
        quad = np.column_stack([rng.uniform(0.1, 1.5, 4), rng.uniform(-1, 1, 4), rng.uniform(-1, 1, 4),
                                rng.uniform(0.1, 1.5, 4)])
        out.append(I.riemann2d(nx, quad, scheme=scheme, ny=ny))
    return out


@pytest.mark.parametrize("scheme", [I.TENO5, I.WENO5JS, I.TENO6])
def test_ensemble_fp64_members_match_oracle(scheme):
    mem = small_members(scheme)
    ens = osbli.Ensemble([c for c, _ in mem], precision=osbli.OSBLI_FP64)
    for p, (_, U) in enumerate(mem):
        ens.set_state(p, U)
    ens.step(12)
    for p, (cfg, U) in enumerate(mem):
        o = O.Oracle(cfg)
        o.set_state(U)
        o.step(12)
        assert relerr(ens.get_state(p), o.get_state()) <= 1e-11, p


@pytest.mark.parametrize("precision,steps,tol", [(osbli.OSBLI_FP64, 15, 0.0), (osbli.OSBLI_MIXED, 1, 1e-7)])
def test_ensemble_members_match_single_handles(precision, steps, tol):
    mem = small_members()
    ens = osbli.Ensemble([c for c, _ in mem], precision=precision)
    for p, (_, U) in enumerate(mem):
        ens.set_state(p, U)
    ens.step(steps)
    worst = 0.0
    for p, (cfg, U) in enumerate(mem):
        s = osbli.Solver(cfg, precision=precision)
        s.set_state(U)
        s.step(steps)
        worst = max(worst, relerr(ens.get_state(p), s.get_state()))
        s.close()
    assert worst <= tol


def test_ensemble_mixed_against_oracle_discontinuous():
    mem = small_members()
    ens = osbli.Ensemble([c for c, _ in mem], precision=osbli.OSBLI_MIXED)
    for p, (_, U) in enumerate(mem):
        ens.set_state(p, U)
    ens.step(20)
    for p, (cfg, U) in enumerate(mem):
        o = O.Oracle(cfg)
        o.set_state(U)
        o.step(20)
        assert l2rel(ens.get_state(p), o.get_state()) <= 1e-4, p   # discontinuous data, as Sod


def test_chunk_and_autotune_are_bitwise_neutral():
    mem = small_members()
    ref = None
    for chunk in (0, 4, 64, "auto"):
        ens = osbli.Ensemble([c for c, _ in mem], precision=osbli.OSBLI_MIXED)
        for p, (_, U) in enumerate(mem):
            ens.set_state(p, U)
        if chunk == "auto":
            before = [ens.get_state(p) for p in range(len(mem))]
            c, ms = ens.autotune(reps=2)
            assert c in (0, 8, 16, 32, 64) and ms > 0
            for p in range(len(mem)):                   # state restored
                assert np.array_equal(ens.get_state(p), before[p])
        else:
            ens.set_chunk(chunk)
        ens.step(6)
        got = [ens.get_state(p) for p in range(len(mem))]
        if ref is None:
            ref = got
        else:
            for a, b in zip(got, ref):
                assert np.array_equal(a, b)
        ens.close()


def test_launch_count_independent_of_member_count():
    mem = small_members()
    counts = []
    for k in (1, 3, 6):
        ens = osbli.Ensemble([c for c, _ in mem[:k]], precision=osbli.OSBLI_MIXED)
        for p, (_, U) in enumerate(mem[:k]):
            ens.set_state(p, U)
        ens.step(1)
        counts.append(ens.launches_per_step())
        ens.close()
    assert counts[0] == counts[1] == counts[2]
    assert counts[0] == 3 * 8          # per stage: 2 ghosts, prim, x left + conv, y conv, FP64 fix, update


def test_nonfinite_member_is_named():
    mem = small_members()
    ens = osbli.Ensemble([c for c, _ in mem], precision=osbli.OSBLI_MIXED)
    for p, (_, U) in enumerate(mem):
        V = U.copy()
        if p == 3:
            V[4, 0, 5, 5] = np.nan
        ens.set_state(p, V)
    with pytest.raises(osbli.OsbliError) as e:
        ens.step(1)
    assert e.value.code == osbli.OSBLI_ENONFINITE and "member 3" in str(e.value)
    # the error words were cleared: a clean state steps again
    ens.set_state(3, mem[3][1])
    ens.step(1)


def test_full_seed0_ensemble_steps_and_conserves():
    """The 64-problem seed-0 ensemble (sizes 128..1024) for a few steps: every member finite with
    positive density."""
    mem = I.riemann_ensemble(0)
    ens = osbli.Ensemble([c for c, _ in mem], precision=osbli.OSBLI_MIXED)
    for p, (_, U) in enumerate(mem):
        ens.set_state(p, U)
    ens.step(5)
    for p, (cfg, U) in enumerate(mem):
        V = ens.get_state(p)
        assert np.isfinite(V).all(), p
        assert V[0].min() > 0.0, p


@pytest.mark.parametrize("precision", [osbli.OSBLI_MIXED, osbli.OSBLI_FP64])
@pytest.mark.parametrize("scheme", [I.TENO5, I.WENO5JS])
def test_persistent_step_is_bitwise_the_graph_step(precision, scheme):
    """One cooperative launch for all steps of all members (device tile queue, grid barriers)
    gives bitwise the states of the per-phase graph form, and of several calls in a row."""
    mem = small_members(scheme)
    states = {}
    for mode in (0, 1):
        ens = osbli.Ensemble([c for c, _ in mem], precision=precision)
        for p, (_, U) in enumerate(mem):
            ens.set_state(p, U)
        if mode:
            ens.set_persistent(True)
            ens.step(7)
            ens.step(5)
            assert ens.launches_per_step() == 1 and ens.persistent_grid() >= 148
        else:
            ens.step(12)
        states[mode] = [ens.get_state(p) for p in range(len(mem))]
        ens.close()
    for a, b in zip(states[0], states[1]):
        assert np.array_equal(a, b)


def test_persistent_barrier_timeout_is_reported_and_the_context_stays_usable():
    """A barrier wait limit of one poll makes the first barrier give up (the blocks cannot all
    arrive that fast): the step returns ETIMEOUT without hanging, and the same ensemble then
    steps correctly with the default limit."""
    mem = small_members()
    ens = osbli.Ensemble([c for c, _ in mem], precision=osbli.OSBLI_MIXED)
    for p, (_, U) in enumerate(mem):
        ens.set_state(p, U)
    ens.set_persistent(True, spin_limit=1)
    with pytest.raises(osbli.OsbliError) as e:
        ens.step(3)
    assert e.value.code == osbli.OSBLI_ETIMEOUT
    ens.set_persistent(True)
    for p, (_, U) in enumerate(mem):
        ens.set_state(p, U)
    ens.step(4)
    ref = osbli.Ensemble([c for c, _ in mem], precision=osbli.OSBLI_MIXED)
    for p, (_, U) in enumerate(mem):
        ref.set_state(p, U)
    ref.step(4)
    for p in range(len(mem)):
        assert np.array_equal(ens.get_state(p), ref.get_state(p))
    ens.close()
    ref.close()
