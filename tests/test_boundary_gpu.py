"""The rest of the C ABI on the GPU: solver fields in caller-owned device
memory (acm_create_ext), the stability warning of acm_set_fields, the
Eq. (3.2) velocity error and the Laplace-law diagnostics computed on the
device, each against the oracle or host formulas of the same quantity."""
import math

import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build
from paper_2012_03525_gb300 import workloads as wl
from test_parity_gpu import _smooth, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("needs a GPU")
    build.build()
    acm.load()
    return t


# ------------------------------------------------------------- acm_create_ext
@pytest.mark.parametrize("shape,prec,two_phase", [
    ((70, 90), acm.FP64, False), ((20, 24, 40), acm.FP32_DEV, False),
    ((48, 48), acm.FP32_DEV, True), ((16, 18, 20), acm.FP64, True)])
def test_create_ext_torch_buffers_bitwise(torch, shape, prec, two_phase):
    """Fields in torch-allocated device tensors on a torch stream give the
    same bits as the library's own allocation; the tensors hold the state."""
    dim = len(shape)
    rng = np.random.default_rng(31)
    st = [1 + 0.01 * _smooth(rng, shape)] + [0.02 * _smooth(rng, shape) for _ in range(dim)]
    kw = dict(nu=0.05, precision=prec)
    phi = None
    if two_phase:
        kw.update(two_phase=True, sigma=1e-2, W=4.0, M=0.2, dt=0.5 if dim == 3 else 1.0)
        phi = np.tanh(3 * _smooth(rng, shape))
    p = acm.make_params(shape, **kw)
    w = st[3] if dim == 3 else None
    with acm.Solver(p) as s:
        s.set_fields(st[0], st[1], st[2], w, phi)
        s.step(23)
        want = s.fields()
    n = acm.storage_elems(p)
    dt = torch.float64 if prec == acm.FP64 else torch.float32
    used = [True, True, True, dim == 3, two_phase]
    bufs = [torch.full((n,), float("nan"), dtype=dt, device="cuda") if used[f] else None
            for b in range(2) for f in range(5)]
    stream = torch.cuda.Stream()
    ptrs = [None if t is None else t.data_ptr() for t in bufs]
    with acm.Solver(p, ext_fields=ptrs, stream=stream.cuda_stream) as s:
        s.set_fields(st[0], st[1], st[2], w, phi)
        if dim == 2:   # unpadded storage: the tensors hold rho - rho0 and u
            stream.synchronize()
            b = s.current_buffer()
            np.testing.assert_array_equal(bufs[5 * b + 1][:st[1].size].cpu().numpy(),
                                          st[1].astype(np.float64 if prec == acm.FP64
                                                       else np.float32).ravel())
        s.step(23)
        got = s.fields()
    for a, b in zip(want, got):
        if a is not None:
            assert np.array_equal(a, b)


def test_create_ext_rejects_bad_buffers(torch):
    p = acm.make_params((16, 16))
    n = acm.storage_elems(p)
    t = [torch.zeros(n + 64, dtype=torch.float64, device="cuda") for _ in range(6)]
    good = [t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), None, None,
            t[3].data_ptr(), t[4].data_ptr(), t[5].data_ptr(), None, None]
    for bad in ([None] + good[1:],                                    # missing rho'
                good[:3] + [t[0].data_ptr()] + good[4:],              # w in 2D
                [good[0] + 8] + good[1:]):                            # misaligned
        with pytest.raises(acm.AcmError) as e:
            acm.Solver(p, ext_fields=bad)
        assert e.value.status == acm.EINVAL


# --------------------------------------------------------- stability warning
def test_set_fields_warns_on_unstable_initial_field():
    """The decaying-turbulence velocities of the learned-closure workload
    (u_max ~ 0.15, nu = 5e-4) at dt = 1 fail |u|^2 dt <= 2 nu: acm_set_fields
    returns ACM_OK and leaves a warning; at dt = 1/30 it does not."""
    rho, u, v = wl.turbulence2d(64, seed=0, u_rms=0.05)[:3]
    for dt, warn in ((1.0, True), (1.0 / 30, False)):
        with acm.Solver(acm.make_params((64, 64), nu=5e-4, dt=dt)) as s:
            s.set_fields(rho, u, v)
            assert ("expected to be unstable" in s.last_error()) == warn


# --------------------------------------------------------- Eq. (3.2) error
@pytest.mark.parametrize("prec", [acm.FP64, acm.FP32_DEV])
def test_reduce_error_tgv_matches_host_formula(prec):
    """Er_u and Er_v of the 2D TGV after 1000 steps against the closed form
    (Eq. 3.1 decay exp(-2 nu k^2 t)): the device sums equal the host's
    Eq. (3.2) on the same fields, and Er_u = Er_v (Section 3.1)."""
    n, u0, nu, steps = 64, 0.02, 0.01, 1000
    with acm.Solver(acm.make_params((n, n), nu=nu, precision=prec)) as s:
        s.set_fields(*wl.tgv2d(n, u0))
        s.step(steps)
        ue, ve = wl.tgv2d_exact(n, u0, nu, steps)
        er = s.reduce_error(ue, ve)
        rho, u, v, _, _ = s.fields()
    assert er[0] == pytest.approx(rel_l2(u, ue), rel=1e-12)
    assert er[1] == pytest.approx(rel_l2(v, ve), rel=1e-12)
    assert er[2] == 0.0
    # the symmetry of Section 3.1 holds to rounding (FP32: its 6e-8 relative
    # rounding of u against an error of ~1e-3)
    assert er[0] == pytest.approx(er[1], rel=1e-6 if prec == acm.FP64 else 1e-3)
    assert 1e-6 < er[0] < 2e-3


def test_reduce_error_3d():
    n = 24
    state = wl.tgv3d(n, 0.05)
    rng = np.random.default_rng(2)
    refs = [state[k] + 1e-3 * _smooth(rng, state[k].shape) for k in (1, 2, 3)]
    with acm.Solver(acm.make_params((n, n, n), nu=0.02)) as s:
        s.set_fields(*state)
        er = s.reduce_error(*refs)
    for a in range(3):
        den = np.sqrt((refs[a] ** 2).sum())
        want = np.sqrt(((state[1 + a] - refs[a]) ** 2).sum()) / den
        assert er[a] == pytest.approx(want, rel=1e-12)


# --------------------------------------------------------- Laplace diagnostics
def _host_laplace(co, p, rho, phi, cs2, dim, walls=()):
    """The quantities acm_reduce_laplace returns, from the oracle's chemical
    potential (Section 2) on the same phi; wall nodes on ``walls`` axes
    (array axes) are left out."""
    mu = co.chem_pot(p, phi)
    keep = np.ones(phi.shape, bool)
    for ax in walls:
        idx = [slice(None)] * phi.ndim
        idx[ax] = [0, -1]
        keep[tuple(idx)] = False
    ph, m, r = phi[keep], mu[keep], rho[keep]
    A = (0.5 * (1 + ph)).sum()
    reff = math.sqrt(A / math.pi) if dim == 2 else (3 * A / (4 * math.pi)) ** (1 / 3)
    wg = 1 - ph ** 2
    inn, out = ph > 0.95, ph < -0.95
    return np.array([A, reff, (m * wg).sum() / wg.sum(), m[inn].mean(), m[out].mean(),
                     cs2 * (r[inn].mean() - r[out].mean()),
                     (dim - 1) * p.sigma / (2 * reff), inn.sum()])


def test_reduce_laplace_batch_matches_oracle(oracle_lib):
    """Three uneven drops (one batch), FP64: the device diagnostics equal
    the host's from the oracle's mu; for the initial tanh profile mu_G is the
    curvature term sigma / (2 R) (within 3 %), and it stays within 5 % of
    the Laplace law while the drops relax."""
    co = oracle_lib
    runs = [(64, 15.0, 3e-3), (90, 22.0, 1e-2), (48, 11.0, 5e-3)]
    params = [acm.make_params((n, n), nu=0.1, two_phase=True, sigma=sg, W=4.0, M=0.2)
              for n, _, sg in runs]
    states = [wl.drop2d(n, R, 4.0) for n, R, _ in runs]
    with acm.Solver(params) as s:
        for r, st in enumerate(states):
            s.set_fields(st[0], st[1], st[2], None, st[3], run=r)
        for steps in (0, 300):
            s.step(steps)
            lap = s.reduce_laplace()
            for r, (n, R, sg) in enumerate(runs):
                rho, _, _, _, phi = s.fields(run=r)
                p = co.make_params((n, n), nu=0.1, two_phase=True, sigma=sg, W=4.0, M=0.2)
                want = _host_laplace(co, p, rho, phi, 1.0 / 3.0, 2)
                np.testing.assert_allclose(lap[r], want, rtol=1e-11, atol=1e-15)
                assert lap[r, 2] == pytest.approx(lap[r, 6], rel=0.03 if steps == 0 else 0.05)


@pytest.mark.parametrize("bc", [[0] * 6, [0, 0, 0, 0, 1, 1]])
def test_reduce_laplace_3d_matches_oracle(oracle_lib, bc):
    co = oracle_lib
    shape = (22, 24, 26)
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(*[np.arange(k, dtype=float) for k in shape], indexing="ij")
    zc = 0.0 if bc[4] else nz / 2
    phi = -np.tanh(2.0 * (np.sqrt((X - nx / 2) ** 2 + (Y - ny / 2) ** 2 + (Z - zc) ** 2) - 8.0) / 4.0)
    kw = dict(dt=0.5, nu=0.1, bc=bc, two_phase=True, sigma=1e-2, W=4.0, M=0.3, theta_deg=90.0)
    z = np.zeros(shape)
    with acm.Solver(acm.make_params(shape, **kw)) as s:
        s.set_fields(np.ones(shape), z, z, z, phi)
        s.step(20)
        lap = s.reduce_laplace()
        rho, _, _, _, ph = s.fields()
    want = _host_laplace(co, co.make_params(shape, **kw), rho, ph, 1.0 / (3 * 0.25), 3,
                         walls=(0,) if bc[4] else ())
    np.testing.assert_allclose(lap, want, rtol=1e-11, atol=1e-15)


def test_reduce_laplace_rejects_single_phase():
    with acm.Solver(acm.make_params((16, 16))) as s:
        s.set_fields(np.ones((16, 16)), np.zeros((16, 16)), np.zeros((16, 16)))
        with pytest.raises(acm.AcmError) as e:
            s.reduce_laplace()
        assert e.value.status == acm.EINVAL


# ------------------------------------------------------------- acm_set_stream
def test_stream_switch_keeps_queued_work_first(torch):
    """A handle moved from one caller stream to another with steps still
    queued on the first: those steps run before the ones queued on the
    second (the library orders the streams on the device), so the result
    is bit for bit one uninterrupted run."""
    shape = (256, 512)
    rng = np.random.default_rng(5)
    st = [1 + 0.01 * _smooth(rng, shape), 0.02 * _smooth(rng, shape), 0.02 * _smooth(rng, shape)]
    p = acm.make_params(shape, nu=0.05, precision=acm.FP32_DEV)
    with acm.Solver(p) as s:
        s.set_fields(*st)
        s.step(600)
        want = s.fields()
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    with acm.Solver(p) as s:
        s.set_stream(a.cuda_stream)
        s.set_fields(*st)
        s.step(300)
        s.set_stream(b.cuda_stream)  # no host wait in between
        s.step(300)
        got = s.fields()
    for k in range(3):
        np.testing.assert_array_equal(got[k], want[k])
