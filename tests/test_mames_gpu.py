"""The MAMEs predictor-corrector (Eqs. 2.6-2.9) on the GPU, the comparison
scheme of Section 3: parity with the oracle in FP64 (1e-12) and FP32
storage, batches, and the paper's comparisons with the simplified scheme
(errors of the 2D Taylor-Green vortex at t = 8; the smaller stable region)."""
import math

import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build
from paper_2012_03525_gb300 import workloads as wl
from test_parity_gpu import _smooth, assert_parity, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    acm.load()


def _both(oracle_lib, shape, state, nsteps, prec=acm.FP64, **kw):
    co = oracle_lib
    rho, u, v = [x.copy() for x in state]
    co.step_mames(co.make_params(shape, **kw), rho, u, v, nsteps=nsteps)
    with acm.Solver(acm.make_params(shape, precision=prec, scheme=acm.SCHEME_MAMES, **kw)) as s:
        s.set_fields(*state)
        s.step(nsteps)
        got = list(s.fields())
    return [rho, u, v, None, None], got


@pytest.mark.parametrize("shape", [(40, 52), (64, 64), (33, 45), (16, 100)])
def test_mames_fp64_matches_oracle(oracle_lib, shape):
    rng = np.random.default_rng(5)
    state = [1 + 0.002 * _smooth(rng, shape), 0.05 * _smooth(rng, shape),
             0.05 * _smooth(rng, shape)]
    ref, got = _both(oracle_lib, shape, state, 200, nu=0.04)
    assert_parity(ref, got)


@pytest.mark.parametrize("dt", [1.0, 0.5])
def test_mames_tgv_fp64_matches_oracle(oracle_lib, dt):
    rho, u, v = wl.tgv2d(50, 0.05, dt=dt)
    ref, got = _both(oracle_lib, (50, 50), [rho, u, v], 300, dt=dt, nu=0.06)
    assert_parity(ref, got)


def test_mames_fp32_deviation(oracle_lib):
    rho, u, v = wl.tgv2d(100, 0.05)
    ref, got = _both(oracle_lib, (100, 100), [rho, u, v], 500, prec=acm.FP32_DEV, nu=0.125)
    assert rel_l2(got[1], ref[1]) < 2e-5
    assert rel_l2(got[0] - 1, ref[0] - 1) < 1e-4


def test_mames_batch_matches_oracle_each(oracle_lib):
    co = oracle_lib
    shapes = [(32, 48), (50, 50), (17, 70)]
    rng = np.random.default_rng(9)
    states = [[1 + 0.002 * _smooth(rng, sh), 0.04 * _smooth(rng, sh), 0.04 * _smooth(rng, sh)]
              for sh in shapes]
    params = [acm.make_params(sh, nu=0.05, scheme=acm.SCHEME_MAMES) for sh in shapes]
    with acm.Solver(params) as s:
        for r, st in enumerate(states):
            s.set_fields(*st, run=r)
        s.step(120)
        for r, (sh, st) in enumerate(zip(shapes, states)):
            rho, u, v = [x.copy() for x in st]
            co.step_mames(co.make_params(sh, nu=0.05), rho, u, v, nsteps=120)
            assert_parity([rho, u, v, None, None], list(s.fields(run=r)))


def test_paper_tgv_errors_and_stability_on_gpu():
    """Section 3.1 on the GPU, FP64: Re = 20, N_L = 50, c = 20: at t = 8 the
    simplified scheme's error is O(1e-3), the MAMEs' O(1e-2); at c = 16 the
    simplified scheme runs and the MAMEs blow up (reported as unstable)."""
    n, c = 100, 20.0
    L, u0 = n / 2, 1.0 / c
    nu = u0 * L / 20.0
    steps = int(8 * L / u0)
    err = {}
    for scheme in (acm.SCHEME_SMAMES, acm.SCHEME_MAMES):
        rho, u, v = wl.tgv2d(n, u0)
        with acm.Solver(acm.make_params((n, n), nu=nu, scheme=scheme)) as s:
            s.set_fields(rho, u, v)
            s.step(steps)
            ue, _ = wl.tgv2d_exact(n, u0, nu, steps)
            err[scheme] = rel_l2(s.fields()[1], ue)
    assert 5e-4 < err[acm.SCHEME_SMAMES] < 5e-3
    assert 3e-3 < err[acm.SCHEME_MAMES] < 3e-2
    c = 16.0
    u0 = 1.0 / c
    nu = u0 * L / 20.0
    outcome = {}
    for scheme in (acm.SCHEME_SMAMES, acm.SCHEME_MAMES):
        rho, u, v = wl.tgv2d(n, u0)
        with acm.Solver(acm.make_params((n, n), nu=nu, scheme=scheme)) as s:
            s.set_fields(rho, u, v)
            s.step(int(2 * L / u0))
            try:
                s.sync()
                f = s.fields()[1]
                outcome[scheme] = bool(np.abs(f).max() < 10 * u0)
            except acm.AcmError as e:
                assert e.status == acm.EUNSTABLE
                outcome[scheme] = False
    assert outcome == {acm.SCHEME_SMAMES: True, acm.SCHEME_MAMES: False}
