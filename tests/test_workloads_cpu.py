"""Pins of the seeded input generators shared by the oracle runs, the GPU
tests and the benchmark: each set-up against its closed-form definition or
the parameters the paper states (Sections 3.1-3.4) and the batch recipe."""
import math

import numpy as np
import pytest

from paper_2012_03525_gb300 import workloads as wl


def _dc(f, axis):
    """centred difference (f_{+1} - f_{-1}) / 2 on a periodic axis"""
    return 0.5 * (np.roll(f, -1, axis) - np.roll(f, 1, axis))


def test_tgv2d_is_discretely_divergence_free_and_matches_its_exact_form():
    n, u0 = 64, 0.05
    rho, u, v = wl.tgv2d(n, u0)
    # cos/sin products: the centred divergence cancels term by term (to rounding
    # of the O(u0 sin k) differences)
    assert np.abs(_dc(u, 1) + _dc(v, 0)).max() < 1e-15 * u0
    ue, ve = wl.tgv2d_exact(n, u0, nu=0.01, t=0.0)
    assert np.array_equal(u, ue) and np.array_equal(v, ve)
    # rho = p / c_s^2 with the pressure's zero-mean cosines (c_s^2 = 1/3 at dt = 1)
    assert abs(rho.mean() - 1.0) < 1e-15
    assert math.isclose(rho.max() - rho.min(), u0 * u0 / (4 / 3) * 4, rel_tol=1e-12)
    # decay exp(-2 nu k^2 t)
    ue, _ = wl.tgv2d_exact(n, u0, nu=0.01, t=100.0)
    k = 2 * np.pi / n
    assert np.allclose(ue, u * math.exp(-2 * 0.01 * k * k * 100.0), rtol=0, atol=1e-17)


def test_tgv3d_is_discretely_divergence_free_with_mean_density_rho0():
    n, u0 = 16, 0.05
    rho, u, v, w = wl.tgv3d(n, u0)
    assert not w.any()
    div = _dc(u, 2) + _dc(v, 1) + _dc(w, 0)
    assert np.abs(div).max() < 1e-15 * u0
    assert abs(rho.mean() - 1.0) < 1e-15
    # p - p0 = rho0 u0^2/16 (cos 2x + cos 2y)(cos 2z + 2): extremes 6 and -2 (x u0^2/16 / c_s^2)
    scale = u0 * u0 / 16 / (1 / 3)
    assert math.isclose(rho.max() - 1.0, 6 * scale, rel_tol=1e-12)


def test_tgv3d_viscosity_matches_the_bench_reading():
    # Re = u0 L / nu with L = n / (2 pi): 256^3, u0 = 0.05, Re = 1600 -> 1.27e-3
    assert math.isclose(wl.tgv3d_nu(256, 0.05, 1600.0), 0.05 * 256 / (2 * np.pi) / 1600.0)
    assert abs(wl.tgv3d_nu(256, 0.05, 1600.0) - 1.273e-3) < 1e-6


def test_drop_batch_recipe():
    runs = wl.batch_drops(512)
    assert runs == wl.batch_drops(512)  # seeded
    n = np.array([r.n for r in runs])
    ratio = np.array([r.radius / r.n for r in runs])
    eps = np.array([r.eps for r in runs])
    sig = np.array([r.sigma for r in runs])
    assert n.min() >= 64 and n.max() <= 512
    assert ratio.min() >= 0.15 and ratio.max() <= 0.35
    assert eps.min() >= 0.0 and eps.max() <= 0.10
    assert sig.min() >= 1e-4 and sig.max() <= 1e-2
    assert all(r.W == 4.0 and r.nu == 0.1 and r.M == 0.1 for r in runs)
    # E[N^2] for N uniform on [64, 512] is about 9.95e4, so ~5.1e7 nodes in 512 runs
    en2 = np.mean(np.arange(64, 513) ** 2)
    assert abs((n * n).sum() / (512 * en2) - 1.0) < 0.06
    assert 4.8e7 < (n * n).sum() < 5.4e7
    # sigma log-uniform: log10 sigma has mean -3 and the variance of U(-4, -2)
    ls = np.log10(sig)
    assert abs(ls.mean() + 3.0) < 0.08 and abs(ls.var() - 1 / 3) < 0.05


def test_drop_profile_is_the_tanh_interface():
    n, R, W = 128, 30.0, 4.0
    rho, u, v, phi = wl.drop2d(n, R, W)
    c = (n - 1) / 2.0
    assert phi[int(c), int(c)] > 0.999 and phi[0, 0] < -0.999
    # phi = -tanh(2 (r - R) / W) along a row through the centre
    x = np.arange(n) - c
    row = phi[64, :]
    r = np.hypot(x, 64 - c)
    assert np.allclose(row, -np.tanh(2 * (r - R) / W), atol=1e-15)
    assert not u.any() and not v.any() and (rho == 1).all()
    # elliptical perturbation R (1 + eps cos 2 theta): longer along x than along y
    _, _, _, pe = wl.drop2d(n, R, W, eps=0.1)
    assert (pe[64, :] > 0).sum() > (pe[:, 64] > 0).sum()


def test_turbulence_is_solenoidal_with_the_requested_rms_and_peak():
    n = 128
    rho, u, v = wl.turbulence2d(n, seed=3)
    assert (rho == 1).all()
    assert math.isclose(np.sqrt(np.mean(u * u + v * v)), 0.05, rel_tol=1e-12)
    # spectral divergence vanishes
    k = np.fft.fftfreq(n) * 2 * np.pi
    KX, KY = np.meshgrid(k, k, indexing="xy")
    div = KX * np.fft.fft2(u) + KY * np.fft.fft2(v)
    assert np.abs(div).max() < 1e-9 * np.abs(np.fft.fft2(u)).max()
    # shell energy peaks near k0 = 8, where k^4 exp(-2 (k/k0)^2) is largest
    kk = np.hypot(*np.meshgrid(np.fft.fftfreq(n) * n, np.fft.fftfreq(n) * n, indexing="xy"))
    e = np.abs(np.fft.fft2(u)) ** 2 + np.abs(np.fft.fft2(v)) ** 2
    shells = np.bincount(np.rint(kk).astype(int).ravel(), e.ravel())
    assert 6 <= int(np.argmax(shells)) <= 10
    # seeded and seed-dependent
    assert np.array_equal(u, wl.turbulence2d(n, seed=3)[1])
    assert not np.array_equal(u, wl.turbulence2d(n, seed=4)[1])


def test_dpsl_setup_and_lattice_parameters():
    n = 320
    rho, u, v = wl.dpsl(n)
    y = np.arange(n) / n
    # shear layers at y = 1/4 and 3/4, perturbation delta_p sin(2 pi (x + 1/4))
    assert abs(u[n // 4, 0]) < 1e-15 and abs(u[3 * n // 4, 0]) < 1e-15
    assert math.isclose(u[n // 2, 0], math.tanh(80 * 0.25))
    assert math.isclose(np.abs(v).max(), 0.05, rel_tol=1e-12)
    assert np.allclose(v[0], 0.05 * np.sin(2 * np.pi * (y + 0.25)))
    # Section 3.3: 320^2, 16000 steps to t = 1, Re = 1e4 -> u_lat = 0.02, nu_lat = 6.4e-4
    us, nu = wl.dpsl_lattice(320, 16000, 1e4)
    assert math.isclose(us, 0.02) and math.isclose(nu, 6.4e-4)


def test_cavity_setup_and_viscosity():
    rho, u, v = wl.cavity2d(16, 0.1)
    assert (u[-1, 1:-1] == 0.1).all() and u[-1, 0] == 0 and u[-1, -1] == 0
    assert not u[:-1].any() and not v.any() and (rho == 1).all()
    # nu = U (n - 1) / Re: 1024^2, lid 0.1, Re = 1000 -> 0.1023
    assert math.isclose(wl.cavity_nu(1024, 0.1, 1000.0), 0.1023)


@pytest.mark.parametrize("n_l,c,re", [(64, 6, 1000.0), (128, 24, 4000.0)])
def test_capillary_wave_parameters_reproduce_the_dimensionless_groups(n_l, c, re):
    cw = wl.CapillaryWave(n_l=n_l, c=c, re=re, cn=4.0 / n_l)
    # Section 3.4: U_c = sigma / (rho0 nu), Re = sigma L / (rho0 nu^2), Cn = W / L,
    # Pe = U_c L^2 / (M sigma), N_t = c N_L steps per T_c
    assert math.isclose(cw.sigma / cw.nu, cw.u_c)
    assert math.isclose(cw.sigma * n_l / cw.nu ** 2, re)
    assert math.isclose(cw.W / n_l, cw.cn)
    assert math.isclose(cw.u_c * n_l ** 2 / (cw.M * cw.sigma), cw.pe)
    assert math.isclose(cw.steps_per_tc * cw.u_c, n_l)
    rho, u, v, phi = cw.initial()
    assert phi.shape == (n_l + 1, n_l)
    # interface at mid-height displaced by A cos(k (x + L/2)): phi < 0 below, > 0 above
    assert (phi[0] < 0).all() and (phi[-1] > 0).all()
