"""Seeded synthetic initial conditions shared by the tests, the oracle runs and
the benchmark.

This module holds only problem set-ups (closed-form initial fields and seeded
random parameters); none of the scheme's arithmetic lives here.  All arrays are
NumPy float64 in [z][y][x] / [y][x] order (x fastest), in lattice units
(delta_x = 1).  Density is absolute; ``p = rho c_s^2`` (Section 2).
"""
from __future__ import annotations

import dataclasses

import numpy as np

BATCH_SEED = 20201207
TURB_TRAIN_SEEDS = range(0, 200)
TURB_TEST_SEEDS = range(1000, 1020)


def cs2_of(dt: float) -> float:
    """c = delta_x / delta_t with delta_x = 1, c_s^2 = c^2 / 3 (Section 2)."""
    return (1.0 / dt) ** 2 / 3.0


def tgv2d(n: int, u0: float, dt: float = 1.0, rho0: float = 1.0, x0: float = 0.0):
    """2D Taylor-Green vortex on an n x n periodic grid, wavenumber k = 2 pi / n
    (the paper's Eqs. 3.1a-c with L = n/2 lattice units, evaluated at t = 0):
      u = -u0 cos(kx) sin(ky), v = u0 sin(kx) cos(ky),
      p = p0 - rho0 u0^2/4 (cos 2kx + cos 2ky),  rho = p / c_s^2, p0 = rho0 c_s^2.
    ``x0`` shifts the node positions (x_i = x0 + i)."""
    k = 2.0 * np.pi / n
    x = x0 + np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")  # arrays [y][x]
    u = -u0 * np.cos(k * X) * np.sin(k * Y)
    v = u0 * np.sin(k * X) * np.cos(k * Y)
    rho = rho0 - rho0 * u0 * u0 / (4.0 * cs2_of(dt)) * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    return rho, u, v


def tgv2d_exact(n: int, u0: float, nu: float, t: float, x0: float = 0.0):
    """Closed-form velocity of the 2D TGV at time t (decay exp(-2 nu k^2 t))."""
    k = 2.0 * np.pi / n
    x = x0 + np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")
    f = np.exp(-2.0 * nu * k * k * t)
    return -u0 * np.cos(k * X) * np.sin(k * Y) * f, u0 * np.sin(k * X) * np.cos(k * Y) * f


def tgv3d(n: int, u0: float, dt: float = 1.0, rho0: float = 1.0):
    """Standard 3D Taylor-Green vortex on an n^3 periodic grid, k = 2 pi / n:
      u = u0 sin(kx) cos(ky) cos(kz), v = -u0 cos(kx) sin(ky) cos(kz), w = 0,
      p = p0 + rho0 u0^2/16 (cos 2kx + cos 2ky)(cos 2kz + 2).
    Arrays are [z][y][x]."""
    k = 2.0 * np.pi / n
    x = np.arange(n, dtype=np.float64) * k
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    rho = rho0 + rho0 * u0 * u0 / (16.0 * cs2_of(dt)) * (np.cos(2 * X) + np.cos(2 * Y)) * (
        np.cos(2 * Z) + 2.0)
    return rho, u, v, w


def tgv3d_nu(n: int, u0: float, re: float) -> float:
    """nu for Re = u0 L / nu with L = n / (2 pi) lattice units."""
    return u0 * (n / (2.0 * np.pi)) / re


def cavity2d(n: int, lid: float):
    """Lid-driven cavity at rest (u = v = 0, rho = 1) with the lid row moving."""
    rho = np.ones((n, n))
    u = np.zeros((n, n))
    v = np.zeros((n, n))
    u[-1, 1:-1] = lid
    return rho, u, v


def cavity_nu(n: int, lid: float, re: float) -> float:
    """nu = U_lid L / Re with the wall-to-wall length L = n - 1."""
    return lid * (n - 1) / re


def drop2d(n: int, radius: float, W: float = 4.0, eps: float = 0.0, cx=None, cy=None):
    """phi = -tanh(2 (r - R(theta)) / W) with R(theta) = R (1 + eps cos 2 theta):
    +1 inside the drop, -1 outside.  Fluid at rest, rho = 1."""
    cx = (n - 1) / 2.0 if cx is None else cx
    cy = (n - 1) / 2.0 if cy is None else cy
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")
    dx, dy = X - cx, Y - cy
    r = np.hypot(dx, dy)
    th = np.arctan2(dy, dx)
    rt = radius * (1.0 + eps * np.cos(2.0 * th))
    phi = -np.tanh(2.0 * (r - rt) / W)
    return np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)), phi


@dataclasses.dataclass
class DropRun:
    n: int
    radius: float
    eps: float
    sigma: float
    W: float = 4.0
    nu: float = 0.1
    M: float = 0.1


def batch_drops(nruns: int = 512, seed: int = BATCH_SEED, nmin: int = 64, nmax: int = 512):
    """Seeded parameters of the batched static/oscillating drop workload:
    grid side N uniform in [nmin, nmax], R = r N with r ~ U[0.15, 0.35],
    elliptical perturbation eps ~ U[0, 0.10], sigma log-uniform in [1e-4, 1e-2],
    W = 4, nu = 0.1, M = 0.1 (lattice units)."""
    rng = np.random.default_rng(seed)
    runs = []
    for _ in range(nruns):
        n = int(rng.integers(nmin, nmax + 1))
        r = float(rng.uniform(0.15, 0.35))
        eps = float(rng.uniform(0.0, 0.10))
        sigma = float(10.0 ** rng.uniform(-4.0, -2.0))
        runs.append(DropRun(n=n, radius=r * n, eps=eps, sigma=sigma))
    return runs


def turbulence2d(n: int, seed: int, u_rms: float = 0.05, k0: float = 8.0):
    """Decaying-turbulence initial field: stream function with random phases and
    energy spectrum E(k) ~ k^4 exp(-2 (k/k0)^2) (k in units of the box
    wavenumber), u = d psi/dy, v = -d psi/dx (divergence free), scaled to the
    requested u_rms, rho = 1."""
    rng = np.random.default_rng(seed)
    kx = np.fft.fftfreq(n) * n
    KX, KY = np.meshgrid(kx, kx, indexing="xy")
    kk = np.hypot(KX, KY)
    kk[0, 0] = 1.0
    ek = kk ** 4 * np.exp(-2.0 * (kk / k0) ** 2)
    # |u_hat|^2 ~ E(k) / (pi k) on the 2D shell -> |psi_hat| = |u_hat| / k
    amp = np.sqrt(ek / (np.pi * kk)) / kk
    amp[0, 0] = 0.0
    phase = np.exp(2j * np.pi * rng.random((n, n)))
    psi_hat = amp * phase
    kxs = 2.0 * np.pi * KX / n
    kys = 2.0 * np.pi * KY / n
    u = np.real(np.fft.ifft2(1j * kys * psi_hat))
    v = np.real(np.fft.ifft2(-1j * kxs * psi_hat))
    s = u_rms / np.sqrt(np.mean(u * u + v * v))
    return np.ones((n, n)), u * s, v * s


def dpsl(n: int, delta_w: float = 80.0, delta_p: float = 0.05):
    """Doubly periodic shear layer on the unit square (Section 3.3, Eqs.
    3.3a-c), n nodes per side at x_i = i / n:
      rho = 1, u = tanh(delta_w (y - 1/4)) for y <= 1/2,
               tanh(delta_w (3/4 - y)) for y > 1/2,
      v = delta_p sin(2 pi (x + 1/4)).
    Velocities in units of the characteristic velocity U = 1."""
    x = np.arange(n, dtype=np.float64) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    u = np.where(Y <= 0.5, np.tanh(delta_w * (Y - 0.25)), np.tanh(delta_w * (0.75 - Y)))
    v = delta_p * np.sin(2 * np.pi * (X + 0.25))
    return np.ones((n, n)), u, v


def dpsl_lattice(n: int, nt: int = 16000, re: float = 1e4):
    """Lattice parameters of the DPSL run with n nodes over L = 1 and nt steps
    per unit time: (velocity scale u_lat per unit U, nu_lat)."""
    dx, dt = 1.0 / n, 1.0 / nt
    return dt / dx, (1.0 / re) * dt / dx ** 2


@dataclasses.dataclass
class CapillaryWave:
    """Lattice parameters of the 2D capillary wave (Section 3.4): unit square,
    N_L nodes per side length L, N_t = c N_L steps per T_c = L / U_c with the
    capillary velocity U_c = sigma / (rho0 nu); Re = sigma L / (rho0 nu^2),
    Cn = W / L, Pe = U_c L^2 / (M sigma).  In lattice units (delta_x =
    delta_t = 1): U_c = 1 / c, nu = U_c N_L / Re, sigma = U_c nu,
    W = Cn N_L, M = U_c N_L^2 / (Pe sigma).  The grid is N_L periodic columns
    by N_L + 1 rows, the first and last rows being the no-slip walls."""
    n_l: int
    c: float
    re: float
    cn: float
    pe: float = 2e4
    amp: float = 0.01

    @property
    def u_c(self):
        return 1.0 / self.c

    @property
    def nu(self):
        return self.u_c * self.n_l / self.re

    @property
    def sigma(self):
        return self.u_c * self.nu

    @property
    def W(self):
        return self.cn * self.n_l

    @property
    def M(self):
        return self.u_c * self.n_l ** 2 / (self.pe * self.sigma)

    @property
    def steps_per_tc(self):
        return self.c * self.n_l

    @property
    def shape(self):
        return (self.n_l + 1, self.n_l)

    def initial(self):
        """phi = tanh(2 (y - h(x)) / W), h(x) = L/2 + A_p L cos(k (x + L/2)),
        fluid at rest, rho = 1 (phi = +1 in the upper half)."""
        L = self.n_l
        x = np.arange(L, dtype=np.float64)
        y = np.arange(L + 1, dtype=np.float64)
        X, Y = np.meshgrid(x, y, indexing="xy")
        h = 0.5 * L + self.amp * L * np.cos(2.0 * np.pi / L * (X + 0.5 * L))
        phi = np.tanh(2.0 * (Y - h) / self.W)
        z = np.zeros(self.shape)
        return np.ones(self.shape), z, z.copy(), phi


def wall_cap(nx: int, ny: int, radius: float, theta_deg: float, W: float = 4.0, xc=None):
    """2D drop sitting on the wall row y = 0 as a circular cap of radius R
    meeting the wall at the contact angle theta (measured inside the drop,
    phi = +1): centre at (xc, -R cos theta), phi = -tanh(2 (r - R) / W).
    Fluid at rest, rho = 1."""
    xc = (nx - 1) / 2.0 if xc is None else xc
    yc = -radius * np.cos(np.radians(theta_deg))
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    X, Y = np.meshgrid(x, y, indexing="xy")
    phi = -np.tanh(2.0 * (np.hypot(X - xc, Y - yc) - radius) / W)
    return np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)), phi


@dataclasses.dataclass
class DropJumping:
    """Coalescence-induced drop jumping on a nonwetting wall (Section 3.7):
    two drops of radius R = N_L centred at (+-R, 0, R) in the box
    [-3R, 3R]^2 x [0, 5R], theta = 180 degrees, simulated on the quarter
    [0, 3R]^2 x [0, 5R] with symmetry planes on the x and y faces (3 N_L x
    3 N_L x 5 N_L nodes) and walls on the z faces.  Re = 1 / Oh^2 (the
    paper's Re = sigma R / (rho0 nu^2), i.e. U_c = sigma / (rho0 nu) as in
    Section 3.4), so in lattice units U_c = 1 / c, nu = U_c N_L / Re,
    sigma = U_c nu, W = Cn N_L, M = U_c N_L^2 / (Pe sigma); results are
    scaled by the capillary-inertial U_ci = sqrt(sigma / (rho0 R)) and
    T_ci = R / U_ci."""
    oh: float
    n_l: int = 40
    c: float = 10.0
    cn: float = 0.1
    pe: float = 8e3

    @property
    def u_c(self):
        return 1.0 / self.c

    @property
    def re(self):
        return 1.0 / self.oh ** 2

    @property
    def nu(self):
        return self.u_c * self.n_l / self.re

    @property
    def sigma(self):
        return self.u_c * self.nu

    @property
    def W(self):
        return self.cn * self.n_l

    @property
    def M(self):
        return self.u_c * self.n_l ** 2 / (self.pe * self.sigma)

    @property
    def u_ci(self):
        return float(np.sqrt(self.sigma / self.n_l))

    @property
    def t_ci(self):
        return self.n_l / self.u_ci

    @property
    def shape(self):
        return (5 * self.n_l, 3 * self.n_l, 3 * self.n_l)

    bc = (4, 4, 4, 4, 1, 1)  # symmetry x, y faces; walls z
    theta_deg = 180.0

    def initial(self):
        """phi = -tanh(2 (r - R) / W), r the distance to the drop centre
        (R, 0, R) (its mirror image across x = 0 is the second drop), fluid at
        rest, rho = 1."""
        nz, ny, nx = self.shape
        R = float(self.n_l)
        Z, Y, X = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                              np.arange(nx, dtype=np.float64), indexing="ij")
        r = np.sqrt((X - R) ** 2 + Y ** 2 + (Z - R) ** 2)
        phi = -np.tanh(2.0 * (r - R) / self.W)
        z = np.zeros(self.shape)
        return np.ones(self.shape), z, z.copy(), z.copy(), phi

    def observables(self, w, phi):
        """Drop centroid velocity W_drop / U_ci and height z_c / R (weights
        (1 + phi) / 2), and the height h_b / R of the drop's lowest point: the
        lowest crossing of phi = 0 over all x-y columns, linearly
        interpolated (0 while the drop touches the wall plane)."""
        nz = phi.shape[0]
        wt = 0.5 * (1.0 + phi)
        zs = np.arange(nz, dtype=np.float64)[:, None, None]
        wd = float((w * wt).sum() / wt.sum())
        zc = float((zs * wt).sum() / wt.sum())
        pos = phi > 0
        has = pos.any(axis=0)
        k = np.argmax(pos, axis=0)[has]
        if k.size == 0:
            hb = float("nan")
        else:
            cols = np.nonzero(has)
            f1 = phi[k, cols[0], cols[1]]
            f0 = phi[np.maximum(k - 1, 0), cols[0], cols[1]]
            zb = np.where(k > 0, (k - 1) + (-f0) / (f1 - f0 + 1e-300), 0.0)
            hb = float(zb.min())
        return wd / self.u_ci, zc / self.n_l, hb / self.n_l
