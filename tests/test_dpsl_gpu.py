"""Doubly periodic shear layer (Section 3.3): the paper's run at N_L = 320,
N_t = 16000, Re = 1e4 stays stable to t = 1, and it reports that the same
case blows up on a 256^2 grid.  Enstrophy (Eq. 3.4) starts at its analytic
value (4/3) delta_w + O(delta_p^2) and decays."""
import math

import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build
from paper_2012_03525_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    acm.load()


def enstrophy_energy(u, v, n):
    """Eq. 3.4 with centred differences, S = 1, dS = 1/n^2 (physical units)."""
    dx = 1.0 / n
    w = (np.roll(v, -1, 1) - np.roll(v, 1, 1)) / (2 * dx) - (np.roll(u, -1, 0) - np.roll(u, 1, 0)) / (2 * dx)
    return 0.5 * (w * w).mean(), 0.5 * (u * u + v * v).mean()


def run_dpsl(n, steps, precision=acm.FP64):
    us, nu = wl.dpsl_lattice(n)
    rho, u, v = wl.dpsl(n)
    s = acm.Solver(acm.make_params((n, n), nu=nu, precision=precision))
    s.set_fields(rho, u * us, v * us)
    return s, us


def test_initial_enstrophy_matches_closed_form():
    n = 320
    _, u, v = wl.dpsl(n)
    om, e = enstrophy_energy(u, v, n)
    exact = 4.0 / 3.0 * 80.0 + 0.25 * (2 * math.pi * 0.05) ** 2
    assert om == pytest.approx(exact, rel=0.02)


def test_stable_at_320_to_t1_with_decaying_enstrophy():
    s, us = run_dpsl(320, 16000)
    rho, u, v, _, _ = s.fields()
    om0, e0 = enstrophy_energy(u / us, v / us, 320)
    s.step(16000)
    rho, u, v, _, _ = s.fields()   # raises AcmError on a blow-up
    om1, e1 = enstrophy_energy(u / us, v / us, 320)
    assert np.isfinite(om1) and om1 < om0
    assert 0.95 * e0 < e1 < e0   # kinetic energy decays slowly at Re = 1e4
    s.close()


def test_blows_up_at_256():
    """Section 3.3: 'Even on a 256 x 256 grid the simulation blowed up'."""
    s, us = run_dpsl(256, 16000)
    s.step(16000)
    with pytest.raises(acm.AcmError) as e:
        s.sync()
    assert e.value.status == acm.EUNSTABLE
    s.close()


def test_dpsl_small_grid_parity(oracle_lib):
    co = oracle_lib
    n = 64
    us, nu = wl.dpsl_lattice(n, nt=3200)
    rho, u, v = wl.dpsl(n, delta_w=20.0)
    st = [rho.copy(), u * us, v * us]
    with acm.Solver(acm.make_params((n, n), nu=nu)) as s:
        s.set_fields(*st)
        s.step(300)
        got = s.fields()
    co.step(co.make_params((n, n), nu=nu), st[0], st[1], st[2], nsteps=300)
    for a, b in ((got[1], st[1]), (got[2], st[2]), (got[0], st[0])):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12
