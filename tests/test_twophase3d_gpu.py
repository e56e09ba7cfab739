"""3D two-phase runs on the GPU (D3Q19 isotropic operators; x, y periodic; z
periodic or wetting walls): parity with the oracle in FP64 (1e-12) and FP32,
and the physics the oracle pins fix: the Laplace law of a static 3D drop
(mu0 = sigma / R) and a drop on a wall moving toward its contact angle."""
import math

import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build
from test_parity_gpu import assert_parity, rel_l2, run_both

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    acm.load()


def _drop3d(shape, R, centre, W=4.0, eps=0.0):
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dx, dy, dz = X - centre[2], Y - centre[1], Z - centre[0]
    r = np.sqrt(dx ** 2 + (dy * (1 + eps)) ** 2 + dz ** 2)
    return -np.tanh(2.0 * (r - R) / W)


def _state(shape, phi, amp=2e-3, walls=False):
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = amp * np.sin(2 * np.pi * Y / ny) * np.cos(2 * np.pi * X / nx)
    v = amp * np.cos(2 * np.pi * Z / nz) * np.sin(2 * np.pi * X / nx)
    w = amp * np.sin(2 * np.pi * X / nx) * np.cos(2 * np.pi * Y / ny)
    if walls:
        for a in (u, v, w):
            a[0] = 0.0
            a[-1] = 0.0
    return [np.ones(shape), u, v, w, phi]


@pytest.mark.parametrize("shape,bc,theta", [
    ((20, 24, 28), [0] * 6, 90.0),
    ((17, 22, 33), [0, 0, 0, 0, 1, 1], 60.0),
    ((16, 20, 24), [0, 0, 0, 0, 1, 1], 150.0),
    ((13, 21, 19), [0] * 6, 90.0),                 # odd ny: pairs whose second node is outside
    ((11, 37, 35), [0, 0, 0, 0, 1, 1], 120.0),     # three tile rows, the last one short and odd
])
def test_two_phase_3d_fp64(oracle_lib, shape, bc, theta):
    walls = bc[4] == 1
    centre = (0.0 if walls else shape[0] / 2, shape[1] / 2 - 0.3, shape[2] / 2 + 0.2)
    phi = _drop3d(shape, 7.0, centre, eps=0.1)
    st = _state(shape, phi, walls=walls)
    sigma, nu = 1e-2, 0.1
    ref, got = run_both(oracle_lib, shape, st, 60, nu=nu, bc=bc, two_phase=True, sigma=sigma,
                        W=4.0, M=0.3, theta_deg=theta, g=(0.0, 0.0, -1e-6))
    assert_parity(ref, got)


def test_two_phase_3d_boussinesq_fp64(oracle_lib):
    """The Boussinesq drop force of Section 3.5 in 3D (z walls, gravity along
    -z, r_rho = 1.15): parity with the oracle."""
    shape, bc = (20, 22, 24), [0, 0, 0, 0, 1, 1]
    phi = _drop3d(shape, 6.0, (12.0, 11.0, 12.0))
    st = _state(shape, phi, walls=True)
    ref, got = run_both(oracle_lib, shape, st, 60, nu=0.1, bc=bc, two_phase=True, sigma=1e-2,
                        W=4.0, M=0.3, theta_deg=90.0, g=(0.0, 0.0, -1e-5), rho_ratio=1.15,
                        dt=0.5)
    assert_parity(ref, got)


def test_two_phase_3d_fp32(oracle_lib):
    shape, bc = (17, 22, 33), [0, 0, 0, 0, 1, 1]
    phi = _drop3d(shape, 7.0, (0.0, 11.0, 16.0))
    st = _state(shape, phi, walls=True)
    ref, got = run_both(oracle_lib, shape, st, 100, gpu_kw={"precision": acm.FP32_DEV}, nu=0.1,
                        bc=bc, two_phase=True, sigma=1e-2, W=4.0, M=0.3, theta_deg=120.0)
    assert rel_l2(got[4], ref[4]) < 1e-6
    for k in (1, 2, 3):
        assert rel_l2(got[k], ref[k]) < 1e-4
    assert rel_l2(got[0] - 1, ref[0] - 1) < 1e-3


def _relaxed_mu_ratio(n, R, W, sigma, steps):
    """Relax a static drop; return (mu_core / (sigma / R_eff), mu averaged
    over the interface / mu_core, max |u|)."""
    c = (n - 1) / 2
    phi = _drop3d((n, n, n), R, (c, c, c), W)
    p = acm.make_params((n, n, n), dt=0.5, nu=0.1, two_phase=True, sigma=sigma, W=W, M=2.0)
    with acm.Solver(p) as s:
        z = np.zeros((n, n, n))
        s.set_fields(np.ones((n, n, n)), z, z, z, phi)
        s.step(steps)
        rho, u, v, w, ph = s.fields()
    r_eff = (3 * ((1 + ph) / 2).sum() / (4 * math.pi)) ** (1 / 3)
    a, kappa = 3 * sigma / (4 * W), 3 * sigma * W / 8
    # mu of the relaxed field with the D3Q19 isotropic Laplacian (NumPy)
    vel = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    vel += [(ex, ey, 0) for ex in (1, -1) for ey in (1, -1)]
    vel += [(ex, 0, ez) for ex in (1, -1) for ez in (1, -1)]
    vel += [(0, ey, ez) for ey in (1, -1) for ez in (1, -1)]
    lap = np.zeros_like(ph)
    for e in vel:
        wgt = 1 / 3 if sum(map(abs, e)) == 1 else 1 / 6
        lap += wgt * (np.roll(ph, (-e[2], -e[1], -e[0]), axis=(0, 1, 2)) - ph)
    mu = 4 * a * ph * (ph * ph - 1) - kappa * lap
    Z, Y, X = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    core = np.sqrt((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2) < r_eff / 2
    wgt = 1 - ph ** 2
    mu_core = mu[core].mean()
    umax = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    return mu_core / (sigma / r_eff), (mu * wgt).sum() / wgt.sum() / mu_core, umax


def test_laplace_law_static_drop_3d():
    """A static 3D drop relaxes to uniform mu = mu0 = sigma / R (Gibbs-Thomson:
    the pressure jump 2 sigma / R over the jump of phi, 2).  The diffuse
    interface raises mu0 by a term that falls fast with W/R: measured 1.37
    (W/R = 1/3), 1.17 (1/4), 1.095 (3/16).  Checked here: at W/R = 3/16 mu is
    uniform to 2 % and within 12 % of sigma/R, and W/R = 1/4 lies further
    off.  Lattice speed c = 2 (dt = 1/2): at c = 1 the 3D continuity SAT,
    (1/6) dx^2 Lap(rho) per step, leaves the grid-scale density mode only
    neutrally stable and the surface-tension force drives it (the oracle
    blows up there too)."""
    fine, uniform, umax = _relaxed_mu_ratio(64, 16.0, 3.0, 2e-2, 90000)
    print(f"3D Laplace W/R=3/16: mu0 ratio {fine:.4f}, uniformity {uniform:.4f}, |u| {umax:.2e}")
    assert fine == pytest.approx(1.0, abs=0.12)
    assert uniform == pytest.approx(1.0, abs=0.02)
    assert umax < 1e-4
    coarse, _, _ = _relaxed_mu_ratio(64, 16.0, 4.0, 2e-2, 90000)
    assert coarse - 1.0 > fine - 1.0 > 0.0


@pytest.mark.parametrize("theta,direction", [(45.0, -1), (135.0, +1)])
def test_drop_on_wall_moves_toward_contact_angle_3d(theta, direction):
    """A hemispherical drop (90 degrees) on a wall of contact angle theta
    spreads (theta < 90: the height on the axis falls) or dewets (theta > 90:
    it rises), as in Section 3.6."""
    shape = (32, 64, 64)
    R = 14.0
    phi = _drop3d(shape, R, (0.0, 31.5, 31.5))
    p = acm.make_params(shape, dt=0.5, nu=0.1, bc=[0, 0, 0, 0, 1, 1], two_phase=True,
                        sigma=1e-2, W=4.0, M=0.5, theta_deg=theta)
    with acm.Solver(p) as s:
        z = np.zeros(shape)
        s.set_fields(np.ones(shape), z, z, z, phi)
        s.step(8000)
        ph = s.fields()[4]
    col = 0.25 * (ph[:, 31, 31] + ph[:, 32, 31] + ph[:, 31, 32] + ph[:, 32, 32])
    j = int(np.where(col < 0)[0][0])
    h = j - 1 + col[j - 1] / (col[j - 1] - col[j])
    assert direction * (h - R) > 1.0, h


@pytest.mark.parametrize("theta", [60.0, 135.0])
def test_drop_spreading_dewetting_section_3_6(theta):
    """Section 3.6 in 3D with the paper's parameters (R = N_L = 32, Oh = 0.1,
    Cn = 0.1, Pe = 8e3, full box [-3R, 3R]^2 x [0, 3R], x/y periodic in
    place of the quarter domain's mirror planes) except the lattice speed:
    c = 20 U_c instead of 10 (the 3D step needs c >= 2 per unit of the
    capillary velocity here).  A hemisphere spreads on theta = 60 and dewets
    on theta = 135 until its height on the axis reaches that of the
    spherical cap of the same volume meeting the wall at theta:
    H/R = (1 - cos t) (2 / (2 - 3 cos t + cos^3 t))^(1/3) = 0.737 (60) and
    1.382 (135), within 6 %."""
    R, oh, cn, pe, c_over_u = 32, 0.1, 0.1, 8e3, 20.0
    nx = ny = 6 * R
    nz = 3 * R + 1
    dt = 1.0
    uc = 1.0 / (c_over_u * dt)           # capillary velocity sigma / (rho nu), lattice
    nu = uc * R * oh ** 2                # Re = U_c R / nu = 1 / Oh^2
    sigma = uc * nu
    W = cn * R
    M = uc * R * R / (pe * sigma)
    Z, Y, X = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny) - (ny - 1) / 2,
                          np.arange(nx) - (nx - 1) / 2, indexing="ij")
    phi = -np.tanh(2.0 * (np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - R) / W)
    zero = np.zeros(phi.shape)
    p = acm.make_params((nz, ny, nx), dt=dt, nu=nu, bc=[0, 0, 0, 0, 1, 1], two_phase=True,
                        sigma=sigma, W=W, M=M, theta_deg=theta, precision=acm.FP32_DEV)
    tc = R / uc
    heights = []
    with acm.Solver(p) as s:
        s.set_fields(np.ones(phi.shape), zero, zero, zero, phi)
        for _ in range(6):
            s.step(int(5 * tc))
            ph = s.fields()[4]
            c0, c1 = ny // 2 - 1, ny // 2
            col = 0.25 * (ph[:, c0, c0] + ph[:, c0, c1] + ph[:, c1, c0] + ph[:, c1, c1])
            j = int(np.where(col < 0)[0][0])
            heights.append((j - 1 + col[j - 1] / (col[j - 1] - col[j])) / R)
    ct = math.cos(math.radians(theta))
    want = (1 - ct) * (2 / (2 - 3 * ct + ct ** 3)) ** (1 / 3)
    print(f"theta {theta}: H/R every 5 T_c {[round(h, 3) for h in heights]}, cap {want:.3f}")
    if theta < 90:
        assert heights[0] < 1.0
    else:
        assert heights[0] > 1.0
    assert heights[-1] == pytest.approx(want, rel=0.06)
    assert abs(heights[-1] - heights[-2]) < 0.02


def _quarter_state(shape, walls=True, amp=2e-3):
    """A drop centred on the corner of the x and y symmetry planes (on the
    z = 0 wall), a smooth flow whose normal velocity vanishes on the planes
    (and on the walls)."""
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = -np.tanh(2.0 * (np.sqrt(X ** 2 + Y ** 2 + (Z - 2.0) ** 2) - 7.0) / 4.0)
    u = amp * np.sin(np.pi * X / (nx - 1)) * np.cos(np.pi * Y / (ny - 1))
    v = amp * np.cos(np.pi * X / (nx - 1)) * np.sin(np.pi * Y / (ny - 1)) * np.cos(Z)
    w = amp * np.cos(np.pi * X / (nx - 1)) * np.cos(2 * np.pi * Y / (ny - 1))
    if walls:
        for a in (u, v, w):
            a[0] = 0.0
            a[-1] = 0.0
    return [np.ones(shape), u, v, w, phi]


@pytest.mark.parametrize("theta,shape", [(90.0, (16, 18, 20)), (150.0, (16, 18, 20)),
                                         (120.0, (11, 17, 35))])
def test_two_phase_3d_symmetry_planes_fp64(oracle_lib, theta, shape):
    """Symmetry planes on all four x and y faces (the quarter domains of
    Sections 3.6-3.7), wetting z walls, gravity along z: parity with the
    oracle at 1e-12 (also with odd ny and a second x tile)."""
    bc = [4, 4, 4, 4, 1, 1]
    st = _quarter_state(shape)
    ref, got = run_both(oracle_lib, shape, st, 60, nu=0.1, bc=bc, two_phase=True, sigma=1e-2,
                        W=4.0, M=0.3, theta_deg=theta, g=(0.0, 0.0, -1e-5), dt=0.5)
    assert_parity(ref, got)
    # the normal velocity stays zero on its planes
    assert np.all(got[1][:, :, 0] == 0) and np.all(got[1][:, :, -1] == 0)
    assert np.all(got[2][:, 0, :] == 0) and np.all(got[2][:, -1, :] == 0)


def test_two_phase_3d_symmetry_planes_fp32(oracle_lib):
    shape, bc = (16, 18, 20), [4, 4, 4, 4, 1, 1]
    st = _quarter_state(shape)
    ref, got = run_both(oracle_lib, shape, st, 100, gpu_kw={"precision": acm.FP32_DEV}, nu=0.1,
                        bc=bc, two_phase=True, sigma=1e-2, W=4.0, M=0.3, theta_deg=120.0,
                        dt=0.5)
    assert rel_l2(got[4], ref[4]) < 1e-6
    for k in (1, 2, 3):
        assert rel_l2(got[k], ref[k]) < 1e-4


@pytest.mark.parametrize("shape", [(12, 14, 16), (10, 19, 13)])
def test_symmetry_planes_equal_doubled_box_on_gpu(shape):
    """On the GPU too, the quarter domain with symmetry planes equals the
    periodic box of twice the size holding the mirror-symmetric fields."""
    nz, ny, nx = shape
    st = _quarter_state(shape, walls=True)

    def ext(f, odd_axes):
        out = f
        for ax in (1, 2):
            n = out.shape[ax]
            inner = np.flip(np.take(out, range(1, n - 1), axis=ax), axis=ax)
            out = np.concatenate([out, -inner if ax in odd_axes else inner], axis=ax)
        return np.ascontiguousarray(out)

    full = [ext(st[0], ()), ext(st[1], (2,)), ext(st[2], (1,)), ext(st[3], ()), ext(st[4], ())]
    kw = dict(nu=0.1, two_phase=True, sigma=1e-2, W=4.0, M=0.3, theta_deg=120.0,
              g=(0.0, 0.0, -1e-5), dt=0.5)
    with acm.Solver(acm.make_params(shape, bc=[4, 4, 4, 4, 1, 1], **kw)) as s:
        s.set_fields(*st)
        s.step(40)
        q = s.fields()
    with acm.Solver(acm.make_params(full[0].shape, bc=[0, 0, 0, 0, 1, 1], **kw)) as s:
        s.set_fields(*full)
        s.step(40)
        f = s.fields()
    for k in range(5):
        assert np.abs(q[k] - f[k][:, :ny, :nx]).max() < 1e-13, k


def _jump_curve(case, prec, quarters):
    p = acm.make_params(case.shape, dt=1.0, nu=case.nu, bc=list(case.bc), two_phase=True,
                        sigma=case.sigma, W=case.W, M=case.M, theta_deg=case.theta_deg,
                        precision=prec)
    every = int(case.t_ci / 4)
    out = []
    with acm.Solver(p) as s:
        s.set_fields(*case.initial())
        for _ in range(quarters):
            s.step(every)
            s.sync()  # raises on a blow-up
            f = s.fields()
            out.append(case.observables(f[3], f[4]))
    return np.array(out)


def test_drop_jumping_quarter_domain_section_3_7():
    """Section 3.7's coalescence-induced jumping on the quarter domain with
    symmetry planes (reduced to N_L = 16, W = 4 nodes; Oh = 0.037, c = 10,
    Pe = 8e3, theta = 180): the run is stable for 4 T_ci, the coalesced drop
    pushes off the nonwetting wall (W_drop > 0 after coalescence) and its
    centroid rises, and FP32 deviation storage follows FP64."""
    from paper_2012_03525_gb300 import workloads as wl
    case = wl.DropJumping(0.037, n_l=16, cn=0.25)
    c64 = _jump_curve(case, acm.FP64, 16)
    c32 = _jump_curve(case, acm.FP32_DEV, 16)
    wd, zc = c64[:, 0], c64[:, 1]
    assert np.all(wd[4:] > 0)          # upward centroid velocity from t = 1.25 T_ci on
    assert zc[-1] > 1.15 and np.all(np.diff(zc[3:]) > 0)
    assert np.abs(c32[:, 0] - wd).max() < 2e-3
    assert np.abs(c32[:, 1] - zc).max() < 2e-3


def test_drop_jumping_full_size_two_steps(oracle_lib):
    """The benchmark's 3D two-phase workload at its full size (the Section
    3.7 quarter domain, 120 x 120 x 200 with symmetry planes and theta = 180
    walls, Oh = 0.037), in the kernels and launch configuration the
    benchmark times: two steps of the whole grid against the oracle, FP64 at
    1e-12 and FP32 deviation storage at the FP32 bounds of the small cases."""
    from paper_2012_03525_gb300 import workloads as wl
    case = wl.DropJumping(0.037)
    init = list(case.initial())
    kw = dict(dt=1.0, nu=case.nu, bc=list(case.bc), two_phase=True, sigma=case.sigma, W=case.W,
              M=case.M, theta_deg=case.theta_deg)
    ref = [x.copy() for x in init]
    oracle_lib.step(oracle_lib.make_params(case.shape, **kw), *ref, nsteps=2)
    for prec in (acm.FP64, acm.FP32_DEV):
        with acm.Solver(acm.make_params(case.shape, precision=prec, **kw)) as s:
            s.set_fields(*init)
            s.step(2)
            got = list(s.fields())
        if prec == acm.FP64:
            assert_parity(ref, got)
        else:
            assert rel_l2(got[4], ref[4]) < 1e-6
            for k in (1, 2, 3):
                assert rel_l2(got[k], ref[k]) < 1e-4
            assert rel_l2(got[0] - 1, ref[0] - 1) < 1e-3
