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
from test_parity_gpu import assert_parity, rel_l2, run_both, _flow, _smooth

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


# ------------------------------------------------------------ two-phase form
def _drop_state(shape, seed, R=None, flow=True):
    ny, nx = shape
    R = 0.3 * min(shape) if R is None else R
    X, Y = np.meshgrid(np.arange(nx) - (nx - 1) / 2 + 0.3, np.arange(ny) - (ny - 1) / 2 - 0.2)
    phi = -np.tanh(2 * (np.hypot(X, Y * 1.1) - R) / 4.0)
    rng = np.random.default_rng(seed)
    u = _flow(rng, shape) if flow else np.zeros(shape)
    v = _flow(rng, shape) if flow else np.zeros(shape)
    return [np.ones(shape), u, v, phi]


TP = dict(nu=0.1, two_phase=True, sigma=1e-2, W=4.0, M=0.3)


@pytest.mark.parametrize("shape", [(64, 64), (16, 130), (33, 71), (100, 112), (70, 57 + 64)])
def test_line2d_tp_periodic_fp64(oracle_lib, shape):
    """Strips of 56 written columns over 64 held ones: one wrapping strip,
    odd widths and heights, the shortest allowed height (16), a last strip
    of a few columns."""
    st = _drop_state(shape, sum(shape))
    ref, got = run_both(oracle_lib, shape, st, 60, gpu_kw=LINE, **TP)
    assert_parity(ref, got)


def test_line2d_tp_general_instantiation_fp64(oracle_lib):
    """Gravity with the Boussinesq drop force (r_rho = 1.15) selects the
    general instantiation."""
    shape = (72, 96)
    st = _drop_state(shape, 5)
    ref, got = run_both(oracle_lib, shape, st, 60, gpu_kw=LINE, g=(0.0, -1e-5, 0.0),
                        rho_ratio=1.15, **TP)
    assert_parity(ref, got)


def test_line2d_tp_fp32(oracle_lib):
    shape = (96, 128)
    st = _drop_state(shape, 6)
    ref, got = run_both(oracle_lib, shape, st, 200, gpu_kw={"precision": acm.FP32_DEV}, **TP)
    assert rel_l2(got[4], ref[4]) < 1e-6
    for k in (1, 2):
        assert rel_l2(got[k], ref[k]) < 1e-4
    assert rel_l2(got[0] - 1, ref[0] - 1) < 1e-3


def test_line2d_tp_batched_drops_match_oracle(oracle_lib):
    """Runs of the seeded drop batch (uneven grids, different sigma) in one
    handle on the two-phase line kernel: every run equals its oracle run."""
    co = oracle_lib
    spec = wl.batch_drops()
    idx = [i for i in range(len(spec)) if spec[i].n <= 150][:5]
    params, states = [], []
    for i in idx:
        d = spec[i]
        params.append(acm.make_params((d.n, d.n), nu=d.nu, two_phase=True, sigma=d.sigma,
                                      W=d.W, M=d.M))
        rho, u, v, phi = wl.drop2d(d.n, d.radius, d.W, eps=d.eps)
        rng = np.random.default_rng(i)
        states.append([rho, _flow(rng, rho.shape), _flow(rng, rho.shape), phi])
    with acm.Solver(params) as s:
        s.set_tuning(acm.TUNE_LINE2D, 1)
        for r, st in enumerate(states):
            s.set_fields(st[0], st[1], st[2], None, st[3], run=r)
        s.step(40)
        for r, i in enumerate(idx):
            d = spec[i]
            got = list(s.fields(run=r))
            rho, u, v, phi = [x.copy() for x in states[r]]
            co.step(co.make_params((d.n, d.n), nu=d.nu, two_phase=True, sigma=d.sigma, W=d.W,
                                   M=d.M), rho, u, v, None, phi, nsteps=40)
            assert_parity([rho, u, v, None, phi], got)


def test_line2d_tp_matches_tile_kernel_fp32():
    shape = (128, 192)
    st = _drop_state(shape, 8)
    out = []
    for line in (1, 0):
        with acm.Solver(acm.make_params(shape, precision=acm.FP32_DEV, **TP)) as s:
            s.set_tuning(acm.TUNE_LINE2D, line)
            s.set_fields(st[0], st[1], st[2], None, st[3])
            s.step(100)
            out.append(s.fields())
    assert rel_l2(out[0][4], out[1][4]) < 1e-6
    for k in (1, 2):
        assert rel_l2(out[0][k], out[1][k]) < 1e-4


# ------------------------------------------- the measured workloads, full size
def test_line2d_tgv4096_full_size(oracle_lib):
    """The 4096^2 TGV of the 2D throughput measurement (u0 = 0.05, nu =
    0.01) at full size on the line kernel, whose items are 32 rows long
    there (smaller grids get shorter ones): two steps against the oracle,
    FP32 deviation storage (the measured form) at the FP32 bounds and FP64
    at 1e-12."""
    n = 4096
    st = list(wl.tgv2d(n, 0.05))
    ref = [x.copy() for x in st]
    oracle_lib.step(oracle_lib.make_params((n, n), nu=0.01), *ref, nsteps=2)
    ref = ref + [None, None]
    for prec in (acm.FP32_DEV, acm.FP64):
        with acm.Solver(acm.make_params((n, n), nu=0.01, precision=prec)) as s:
            s.set_tuning(acm.TUNE_LINE2D, 1)
            s.set_fields(*st)
            s.step(2)
            got = list(s.fields())
        if prec == acm.FP64:
            assert_parity(ref, got)
        else:
            assert_parity(ref, got, tol=2e-5, tol_rho=1e-4)


@pytest.mark.parametrize("prec", [acm.FP64, acm.FP32_DEV])
def test_line2d_tp_full_drop_batch_sampled(oracle_lib, prec):
    """The whole 512-run batched-drop workload in one handle on the two-phase
    line kernel, in the launch configuration the measurement times (with
    this many runs its items are 64 rows long): after 4 steps, six sampled
    runs (the four largest grids and the two smallest, each given a smooth
    flow) equal their oracle runs, FP64 at 1e-12 and FP32 at the FP32
    bounds of the small cases."""
    co = oracle_lib
    spec = wl.batch_drops()
    order = np.argsort([d.n for d in spec])
    pick = [int(i) for i in list(order[-4:]) + list(order[:2])]
    rng = np.random.default_rng(12)
    states = []
    for i, d in enumerate(spec):
        rho, u, v, phi = wl.drop2d(d.n, d.radius, d.W, eps=d.eps)
        if i in pick:
            u, v = u + _flow(rng, u.shape), v + _flow(rng, v.shape)
        states.append([rho, u, v, phi])
    params = [acm.make_params((d.n, d.n), nu=d.nu, two_phase=True, sigma=d.sigma, W=d.W, M=d.M,
                              precision=prec) for d in spec]
    steps = 4
    with acm.Solver(params) as s:
        s.set_tuning(acm.TUNE_LINE2D, 1)
        for r, st in enumerate(states):
            s.set_fields(st[0], st[1], st[2], None, st[3], run=r)
        s.step(steps)
        got = {i: list(s.fields(run=i)) for i in pick}
    for i in pick:
        d = spec[i]
        st = [x.copy() for x in states[i]]
        co.step(co.make_params((d.n, d.n), nu=d.nu, two_phase=True, sigma=d.sigma, W=d.W, M=d.M),
                st[0], st[1], st[2], None, st[3], nsteps=steps)
        ref = [st[0], st[1], st[2], None, st[3]]
        if prec == acm.FP64:
            assert_parity(ref, got[i])
        else:
            assert rel_l2(got[i][4], ref[4]) < 1e-6
            for k in (1, 2):
                assert rel_l2(got[i][k], ref[k]) < 1e-4
            assert rel_l2(got[i][0] - 1, ref[0] - 1) < 1e-3
