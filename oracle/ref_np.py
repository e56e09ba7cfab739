"""Independent NumPy restatement of the simplified MAME step (periodic grids).

TEST INFRASTRUCTURE ONLY.  It shares nothing with the C oracle: it is written
with whole-array shifts (``np.roll``) instead of index loops, and it exists to
cross-check ``acm_oracle.c`` on small periodic grids.

Section 2 of Huang (arXiv:2012.03525):
  Eq. (2.10)  rho^{n+1} = rho^n - dt d_a(rho u_a)^n + 1/2 cs^2 dt^2 d_aa rho^n
  Eq. (2.11)  (rho u_a)^{n+1} = (rho u_a)^n - dt d_b(rho u_a u_b + rho cs^2 delta_ab)^n
              + nu dt d_bb(rho u_a)^n - (nu + 1/2 cs^2 dt)(d_a rho^{n+1} - d_a rho^n)
              (+ dt rho^{n+1} g_a, + dt F_ST,a for two-phase flows)
  Eq. (2.12)/(2.13)  centred differences and the 5-point Laplacian.
Two-phase: F_ST = -phi grad(mu), mu = 4 a phi(phi^2-1) - kappa Lap(phi),
Eq. (2.14) advanced by Heun RK2 with u^n frozen, D2Q9/D3Q19-weighted
isotropic gradient and Laplacian.
"""
from __future__ import annotations

import itertools

import numpy as np


def _shift(f, axis, s):
    """f(x + s e_axis) on a periodic grid (arrays are [z][y][x] / [y][x])."""
    return np.roll(f, -s, axis=axis)


def _axes(f):
    # physical direction d (0=x, 1=y, 2=z) -> numpy axis
    nd = f.ndim
    return [nd - 1 - d for d in range(nd)]


def ddx(f, d):
    ax = _axes(f)[d]
    return 0.5 * (_shift(f, ax, 1) - _shift(f, ax, -1))


def lap(f):
    out = -2.0 * f.ndim * f
    for ax in _axes(f):
        out = out + _shift(f, ax, 1) + _shift(f, ax, -1)
    return out


def _velocity_set(ndim):
    """Lattice velocities and weights (D2Q9 / D3Q19), c_s^2 = 1/3."""
    vecs, ws = [], []
    for e in itertools.product((-1, 0, 1), repeat=ndim):
        n2 = sum(abs(x) for x in e)
        if ndim == 2:
            w = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}[n2]
        else:
            if n2 == 3:
                continue
            w = {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[n2]
        vecs.append(e)
        ws.append(w)
    return vecs, ws


def _shift_vec(f, e):
    out = f
    for d, s in enumerate(e):
        if s:
            out = _shift(out, _axes(f)[d], s)
    return out


def grad_iso(f, d):
    vecs, ws = _velocity_set(f.ndim)
    out = np.zeros_like(f)
    for e, w in zip(vecs, ws):
        if e[d]:
            out = out + w * e[d] * _shift_vec(f, e)
    return 3.0 * out


def lap_iso(f):
    vecs, ws = _velocity_set(f.ndim)
    out = np.zeros_like(f)
    for e, w in zip(vecs, ws):
        if any(e):
            out = out + w * (_shift_vec(f, e) - f)
    return 6.0 * out


def chem_pot(phi, sigma, W):
    a = 3.0 * sigma / (4.0 * W)
    kappa = 3.0 * sigma * W / 8.0
    return 4.0 * a * phi * (phi * phi - 1.0) - kappa * lap_iso(phi)


def step(rho, vel, nsteps=1, dt=1.0, nu=0.01, g=None, sat_mask=3, phi=None, sigma=0.0,
         W=4.0, M=0.0):
    """Returns (rho, [u, v(, w)], phi) after ``nsteps`` steps (inputs untouched)."""
    rho = rho.copy()
    vel = [x.copy() for x in vel]
    phi = None if phi is None else phi.copy()
    ndim = rho.ndim
    cs2 = (1.0 / dt) ** 2 / 3.0
    g = [0.0] * ndim if g is None else g
    for _ in range(nsteps):
        m = [rho * x for x in vel]
        drho = sum(ddx(m[d], d) for d in range(ndim))
        rho1 = rho - dt * drho
        if sat_mask & 1:
            rho1 = rho1 + 0.5 * cs2 * dt * dt * lap(rho)
        if phi is not None:
            mu = chem_pot(phi, sigma, W)
        new = []
        for a in range(ndim):
            flux = sum(ddx(m[a] * vel[b], b) for b in range(ndim)) + cs2 * ddx(rho, a)
            ma = m[a] - dt * flux + nu * dt * lap(m[a])
            if sat_mask & 2:
                ma = ma - (nu + 0.5 * cs2 * dt) * (ddx(rho1, a) - ddx(rho, a))
            ma = ma + dt * rho1 * g[a]
            if phi is not None:
                ma = ma - dt * phi * grad_iso(mu, a)
            new.append(ma / rho1)
        if phi is not None:
            def rhs(f, muf):
                return -sum(vel[d] * grad_iso(f, d) for d in range(ndim)) + M * lap_iso(muf)
            phis = phi + dt * rhs(phi, mu)
            phi = 0.5 * (phi + phis + dt * rhs(phis, chem_pot(phis, sigma, W)))
        rho, vel = rho1, new
    return rho, vel, phi
