"""Oracle parity of the 2D line-marching kernel (acm_line2d.cu): single-phase
grids periodic on all four faces whose width is a multiple of 64, stepped
one warp per 64-column strip of up to 32 rows.  Strips are checked at the
periodic seam (one strip wrapping onto itself, several strips), with row
counts that leave short last items (not multiples of 32 or of the 4-row
register queue), with rho0 != 1 and a body force (the general
instantiation), in batches of runs of different sizes, in FP64 (1e-12) and
FP32 deviation storage (the kernel is the default for FP32 storage; the
FP64 cases select it with ACM_TUNE_LINE2D); the line and tile kernels agree,
and a blow-up is reported."""
import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build
from paper_2012_03525_gb300 import workloads as wl
from test_parity_gpu import assert_parity, run_both, _smooth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    acm.load()


LINE = {"tuning": {acm.TUNE_LINE2D: 1}}


def _state(shape, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    return [1 + 0.01 * _smooth(rng, shape), amp * _smooth(rng, shape), amp * _smooth(rng, shape)]


@pytest.mark.parametrize("shape", [(64, 64), (37, 128), (100, 192), (5, 64), (4, 256)])
def test_line2d_periodic_random_fp64(oracle_lib, shape):
    st = _state(shape, sum(shape))
    ref, got = run_both(oracle_lib, shape, st, 150, gpu_kw=LINE, nu=0.05)
    assert_parity(ref, got)


@pytest.mark.parametrize("shape", [(70, 128), (33, 64)])
def test_line2d_general_instantiation_fp64(oracle_lib, shape):
    """rho0 != 1 and a body force select the general instantiation."""
    st = _state(shape, 7 + sum(shape))
    st[0] = st[0] * 1.3
    ref, got = run_both(oracle_lib, shape, st, 120, gpu_kw=LINE, nu=0.04, rho0=1.3,
                        g=(1e-5, -2e-5, 0))
    assert_parity(ref, got, rho0=1.3)


def test_line2d_fp32_deviation(oracle_lib):
    shape = (96, 256)
    st = _state(shape, 3)
    ref, got = run_both(oracle_lib, shape, st, 300, gpu_kw={"precision": acm.FP32_DEV},
                        nu=0.05)
    assert_parity(ref, got, tol=2e-5, tol_rho=1e-4)


def test_line2d_batched_runs_of_different_sizes(oracle_lib):
    co = oracle_lib
    specs = [((64, 64), 0.05), ((45, 128), 0.02), ((130, 64), 0.08), ((8, 320), 0.03)]
    params = [acm.make_params(shape, nu=nu) for shape, nu in specs]
    states = [_state(shape, 20 + i) for i, (shape, _) in enumerate(specs)]
    with acm.Solver(params) as s:
        s.set_tuning(acm.TUNE_LINE2D, 1)
        for r, st in enumerate(states):
            s.set_fields(*st, run=r)
        s.step(80)
        for r, (shape, nu) in enumerate(specs):
            got = list(s.fields(run=r))
            rho, u, v = [x.copy() for x in states[r]]
            co.step(co.make_params(shape, nu=nu), rho, u, v, nsteps=80)
            assert_parity([rho, u, v, None, None], got)


@pytest.mark.parametrize("prec", [acm.FP64, acm.FP32_DEV])
def test_line2d_matches_tile_kernel(prec):
    """The two kernels of the same step: FP64 within rounding order (1e-14),
    FP32 within the FP32 tolerance."""
    shape = (256, 512)
    st = list(wl.tgv2d(512, 0.05))
    st = [x[:256] for x in st]
    out = []
    for line in (1, 0):
        with acm.Solver(acm.make_params(shape, nu=0.02, precision=prec)) as s:
            s.set_tuning(acm.TUNE_LINE2D, line)
            s.set_fields(*st)
            s.step(100)
            out.append(s.fields())
    tols = (1e-14, 1e-14, 1e-14) if prec == acm.FP64 else (1e-4, 2e-5, 2e-5)
    for k in range(3):
        a, b = out[0][k] - (1.0 if k == 0 else 0.0), out[1][k] - (1.0 if k == 0 else 0.0)
        assert np.linalg.norm(a - b) <= tols[k] * np.linalg.norm(b), k


def test_line2d_blow_up_reported_as_unstable():
    """No SATs on grid-scale noise blows up; the line kernel's flag makes the
    next synchronising call report ACM_EUNSTABLE."""
    rng = np.random.default_rng(0)
    shape = (64, 128)
    with acm.Solver(acm.make_params(shape, nu=0.0, sat_mask=0)) as s:
        s.set_tuning(acm.TUNE_LINE2D, 1)
        s.set_fields(1 + 0.1 * rng.standard_normal(shape), 0.3 * rng.standard_normal(shape),
                     0.3 * rng.standard_normal(shape))
        s.step(3000)
        with pytest.raises(acm.AcmError) as e:
            s.sync()
        assert e.value.status == acm.EUNSTABLE


def test_line2d_autotune_and_tuning_knob():
    shape = (128, 256)
    st = _state(shape, 9)
    with acm.Solver(acm.make_params(shape, nu=0.05)) as s:
        assert s.get_tuning(acm.TUNE_LINE2D) == 0  # FP64 default: the tile kernel
    with acm.Solver(acm.make_params(shape, nu=0.05, precision=acm.FP32_DEV)) as s:
        assert s.get_tuning(acm.TUNE_LINE2D) == 1
        s.set_fields(*st)
        ms = s.autotune(5)
        assert ms > 0
        assert s.get_tuning(acm.TUNE_LINE2D) in (0, 1)
        with pytest.raises(acm.AcmError):
            s.set_tuning(acm.TUNE_LINE2D, 2)


def test_line2d_tgv64_fp64_1000_steps(oracle_lib):
    """The 64^2 decaying TGV (u0 = 0.02, nu = 0.01) over 1000 steps on the line
    kernel (one strip wrapping onto itself): relative L2 <= 1e-12 against the
    oracle, mass conserved."""
    n, u0, nu, steps = 64, 0.02, 0.01, 1000
    state = list(wl.tgv2d(n, u0))
    ref, got = run_both(oracle_lib, (n, n), state, steps, gpu_kw=LINE, nu=nu)
    assert_parity(ref, got)
    assert abs(got[0].sum() - state[0].sum()) < 1e-12 * state[0].sum()
