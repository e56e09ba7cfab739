"""Two-phase runs with walls on the GPU (Section 2 wall conditions: no-slip
velocity, d_n mu = 0, and the wetting condition d_n phi = -(2/W) cos(theta)
(1 - phi_w^2)).  Parity with the oracle in FP64 (1e-12) and FP32 storage, a
batch of runs with different contact angles, the apparent contact angle a
spreading drop relaxes to, and the capillary-wave periods of Section 3.4,
Table 2."""
import json
import math
import os

import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build
from paper_2012_03525_gb300 import workloads as wl

import twophase_analysis as ta
from test_parity_gpu import assert_parity, rel_l2, run_both

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    acm.load()


def _perturb(state, amp=2e-3):
    """Add a smooth shear u = amp sin(2 pi x / nx) sin(pi y / (ny - 1)) so that
    the advection terms are exercised from the first step."""
    rho, u, v, phi = state
    ny, nx = rho.shape
    u = u + amp * np.sin(2 * np.pi * np.arange(nx) / nx)[None, :] * np.sin(
        np.pi * np.arange(ny) / (ny - 1))[:, None]
    return [rho, u, v, phi]


# (ny, nx), bc, theta, where the drop sits
CASES = [
    ((40, 96), [0, 0, 1, 1, 0, 0], 60.0, "bottom"),     # channel, x periodic
    ((45, 70), [1, 1, 1, 1, 0, 0], 135.0, "corner"),    # closed box, ragged tiles
    ((64, 37), [1, 1, 0, 0, 0, 0], 45.0, "left"),       # walls in x only
    ((33, 33), [1, 1, 1, 1, 0, 0], 90.0, "corner"),     # neutral wetting
]


def _state(shape, where, theta):
    ny, nx = shape
    if where == "bottom":
        st = list(wl.wall_cap(nx, ny, 16.0, theta))
    elif where == "left":
        st = [a.T.copy() for a in wl.wall_cap(ny, nx, 14.0, theta)]
        st[1], st[2] = st[2].copy(), st[1].copy()
    else:  # quarter drop in the corner (0, 0)
        x = np.arange(nx, dtype=np.float64)
        y = np.arange(ny, dtype=np.float64)
        X, Y = np.meshgrid(x, y, indexing="xy")
        phi = -np.tanh(2.0 * (np.hypot(X - 3.0, Y - 2.0) - 15.0) / 4.0)
        st = [np.ones(shape), np.zeros(shape), np.zeros(shape), phi]
    return _perturb(st)


def _zero_wall_velocity(st, bc):
    rho, u, v, phi = st
    for a in (u, v):
        if bc[0]:
            a[:, 0] = 0.0
            a[:, -1] = 0.0
        if bc[2]:
            a[0, :] = 0.0
            a[-1, :] = 0.0
    return st


@pytest.mark.parametrize("shape,bc,theta,where", CASES)
def test_two_phase_walls_fp64(oracle_lib, shape, bc, theta, where):
    st = _zero_wall_velocity(_state(shape, where, theta), bc)
    sigma, nu = 1e-2, 0.1
    ref, got = run_both(oracle_lib, shape, st, 200, nu=nu, bc=bc, two_phase=True, sigma=sigma,
                        W=4.0, M=0.5, theta_deg=theta)
    assert_parity(ref, got)


def test_two_phase_walls_fp32(oracle_lib):
    shape, bc, theta, where = CASES[1]
    st = _zero_wall_velocity(_state(shape, where, theta), bc)
    ref, got = run_both(oracle_lib, shape, st, 300, gpu_kw={"precision": acm.FP32_DEV}, nu=0.1,
                        bc=bc, two_phase=True, sigma=1e-2, W=4.0, M=0.5, theta_deg=theta)
    assert rel_l2(got[4], ref[4]) < 1e-6
    for k in (1, 2):
        assert rel_l2(got[k], ref[k]) < 1e-4
    assert rel_l2(got[0] - 1, ref[0] - 1) < 1e-3


def test_batch_with_different_contact_angles(oracle_lib):
    """One batched launch per step over channels whose walls have different
    contact angles (the wetting coefficient is per run)."""
    co = oracle_lib
    thetas = [30.0, 75.0, 90.0, 120.0, 160.0]
    shapes = [(40, 96), (36, 64), (50, 100), (33, 70), (44, 80)]
    bc = [0, 0, 1, 1, 0, 0]
    params, states = [], []
    for (ny, nx), th in zip(shapes, thetas):
        params.append(acm.make_params((ny, nx), nu=0.1, bc=bc, two_phase=True, sigma=1e-2,
                                      W=4.0, M=0.5, theta_deg=th))
        states.append(_zero_wall_velocity(_perturb(list(wl.wall_cap(nx, ny, 12.0, 90.0))), bc))
    steps = 150
    with acm.Solver(params) as s:
        for r, st in enumerate(states):
            s.set_fields(st[0], st[1], st[2], None, st[3], run=r)
        s.step(steps)
        for r, ((ny, nx), th) in enumerate(zip(shapes, thetas)):
            got = list(s.fields(run=r))
            rho, u, v, phi = [x.copy() for x in states[r]]
            p = co.make_params((ny, nx), nu=0.1, bc=bc, two_phase=True, sigma=1e-2, W=4.0,
                               M=0.5, theta_deg=th)
            co.step(p, rho, u, v, None, phi, nsteps=steps)
            assert_parity([rho, u, v, None, phi], got)


@pytest.mark.parametrize("theta", [60.0, 135.0])
def test_spreading_drop_relaxes_to_contact_angle(theta):
    """Section 3.6 in 2D: a semicircular drop on a wall of contact angle theta
    spreads (60) or dewets (135) until its apparent angle, measured from its
    height and base as a circular cap, is theta within 3 degrees."""
    ny, nx, R = 80, 240, 30.0
    rho, u, v, phi = wl.wall_cap(nx, ny, R, 90.0)
    p = acm.make_params((ny, nx), nu=0.1, bc=[0, 0, 1, 1, 0, 0], two_phase=True, sigma=1e-2,
                        W=4.0, M=0.5, theta_deg=theta)
    with acm.Solver(p) as s:
        s.set_fields(rho, u, v, None, phi)
        angles = []
        for _ in range(6):
            s.step(20000)
            angles.append(ta.cap_angle(s.fields()[4])[0])
        assert np.atleast_2d(s.reduce())[0, 7] == 0
    assert angles[-1] == pytest.approx(theta, abs=3.0), angles
    assert abs(angles[-1] - angles[-2]) < 1.0, angles


def _capillary_period(cw, t_max=60.0):
    p = acm.make_params(cw.shape, nu=cw.nu, bc=[0, 0, 1, 1, 0, 0], two_phase=True,
                        sigma=cw.sigma, W=cw.W, M=cw.M)
    rho, u, v, phi = cw.initial()
    tc = cw.steps_per_tc
    every = max(1, int(tc) // 96)
    ts, hs = [], []
    with acm.Solver(p) as s:
        s.set_fields(rho, u, v, None, phi)
        for it in range(int(t_max * tc) // every + 1):
            f = s.fields()[4]
            ts.append(it * every / tc)
            hs.append((0.5 * cw.n_l - ta.zero_crossing(f[:, 0])) / (cw.amp * cw.n_l))
            if ta.oscillation_period(ts, hs) is not None:
                break
            s.step(every)
    return ta.oscillation_period(ts, hs)


@pytest.mark.parametrize("re,key", [(1000.0, "Re1000"), (4000.0, "Re4000")])
def test_capillary_wave_periods_table2(re, key):
    """Section 3.4, Table 2: the period of the capillary wave (first maximum
    of h~) at N_L = 64, c = 6, Cn = 0.0625 and at N_L = 128, c = 24,
    Cn = 0.03125 (Pe = 2e4).  The coarse period lies within 7 % of the
    analytic one (the paper: 3-3.5 %; measured here 5.3-5.4 %), the fine one
    within 3 % (the paper: 1-1.4 %; measured here 1.7-2.7 %), and refinement
    brings it closer to the analytic period.  The remaining gap to the
    paper's own errors is spatial (it does not move with c or Pe)."""
    tab = GOLDEN["capillary_wave_periods"]
    exact = tab["analytical"][key]
    coarse = _capillary_period(wl.CapillaryWave(n_l=64, c=6, re=re, cn=0.0625))
    fine = _capillary_period(wl.CapillaryWave(n_l=128, c=24, re=re, cn=0.03125))
    print(f"Re={re}: period N_L=64 {coarse:.3f}  N_L=128 {fine:.3f}  analytic {exact}  "
          f"paper {tab['NL64_c6'][key]} / {tab['NL128_c24'][key]}")
    assert coarse == pytest.approx(exact, rel=0.07)
    assert fine == pytest.approx(exact, rel=0.03)
    assert abs(fine - exact) < abs(coarse - exact)


def test_capillary_wave_unstable_at_c5_on_gpu():
    """Section 3.4: the capillary wave (Re = 1000, N_L = 64, Cn = 0.0625,
    Pe = 2e4) blows up at c = 5 -- reported as ACM_EUNSTABLE -- and runs at
    c = 6."""
    out = {}
    for c in (5.0, 6.0):
        cw = wl.CapillaryWave(n_l=64, c=c, re=1000.0, cn=0.0625)
        p = acm.make_params(cw.shape, nu=cw.nu, bc=[0, 0, 1, 1, 0, 0], two_phase=True,
                            sigma=cw.sigma, W=cw.W, M=cw.M)
        with acm.Solver(p) as s:
            s.set_fields(*cw.initial()[:3], None, cw.initial()[3])
            s.step(int(6 * cw.steps_per_tc))
            try:
                s.sync()
                out[c] = bool(np.abs(s.fields()[1]).max() < 1.0)
            except acm.AcmError as e:
                assert e.status == acm.EUNSTABLE
                out[c] = False
    assert out == {5.0: False, 6.0: True}


@pytest.mark.parametrize("prec", [acm.FP64, acm.FP32_DEV])
def test_falling_drop_boussinesq(oracle_lib, prec):
    """Section 3.5's falling drop in a walled 2D box (planar, not
    axisymmetric): the body force acts on the drop only, times
    2 (r - 1)/(r + 1) for r_rho = 1.15.  Parity with the oracle; the drop's
    mean velocity points along g."""
    ny, nx = 96, 40
    rho, u, v, phi = wl.drop2d(max(nx, ny), 10.0, 4.0, cx=nx / 2 - 0.5, cy=ny - 20.0)
    phi = np.ascontiguousarray(phi[:ny, :nx])
    st = [np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), phi]
    kw = dict(nu=0.05, bc=[1, 1, 1, 1, 0, 0], two_phase=True, sigma=5e-3, W=4.0, M=0.2,
              g=(0.0, -1e-4, 0.0), rho_ratio=1.15)
    ref, got = run_both(oracle_lib, (ny, nx), st, 300, gpu_kw={"precision": prec}, **kw)
    if prec == acm.FP64:
        assert_parity(ref, got)
    else:
        # FP32 velocities (relative rounding 6e-8) advect phi for 300 steps;
        # the velocities are the small residual of gravity, pressure and
        # surface tension (measured 1.5e-4; the static-drop FP32 test allows
        # 1e-3 for the same reason)
        assert rel_l2(got[4], ref[4]) < 5e-6
        for k in (1, 2):
            assert rel_l2(got[k], ref[k]) < 1e-3
    inside = got[4] > 0
    assert got[2][inside].mean() < 0 and abs(got[1][inside].mean()) < abs(got[2][inside].mean())
