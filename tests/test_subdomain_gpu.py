"""3D sub-domains on one GPU: a periodic grid split along z into slabs (a 3D
batch whose runs have ACM_BC_HALO z faces) with a halo-copy kernel before
every step gives bit-for-bit the unsplit run, in FP32 and FP64, for even and
uneven slabs, down to two planes per slab, through graph replay and direct
launches; the per-slab diagnostics add up to the whole grid's."""
import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    acm.load()


def _fields(shape, seed=4):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky, kz = 2 * np.pi / nx, 2 * np.pi / ny, 2 * np.pi / nz
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, 3)
    u = 0.05 * np.sin(kx * x + ph[0]) * np.cos(ky * y) * np.cos(kz * z)
    v = -0.05 * np.cos(kx * x) * np.sin(ky * y + ph[1]) * np.cos(kz * z)
    w = 0.02 * np.sin(kz * z + ph[2]) * np.cos(kx * x)
    rho = 1.0 + 1e-3 * np.cos(kx * x + 2 * kz * z)
    return [rho, u, v, w]


def _run(params_list, state, nsteps, z_parts):
    with acm.Solver(params_list) as s:
        z0 = 0
        for r, n in enumerate(z_parts):
            s.set_fields(*[f[z0:z0 + n] for f in state], run=r)
            z0 += n
        s.step(nsteps)
        out = [np.concatenate(parts, axis=0) for parts in
               zip(*[s.fields(run=r)[:4] for r in range(len(z_parts))])]
        red = np.atleast_2d(s.reduce())
    return out, red


@pytest.mark.parametrize("prec", [acm.FP64, acm.FP32_DEV])
@pytest.mark.parametrize("parts", [(40,), (20, 20), (13, 14, 13), (2, 19, 2, 17), (10, 10, 10, 10)])
def test_slabs_equal_unsplit_bitwise(prec, parts):
    shape = (40, 36, 64)
    state = _fields(shape)
    nsteps = 70  # one 64-step graph replay plus direct launches
    kw = dict(nu=0.02, precision=prec)
    ref, red_ref = _run(acm.make_params(shape, **kw), state, nsteps, (shape[0],))
    got, red = _run(acm.subdomain_params(shape, parts, **kw), state, nsteps, parts)
    for k in range(4):
        assert np.array_equal(got[k], ref[k]), (k, float(np.abs(got[k] - ref[k]).max()))
    # diagnostics: sums add up, maxima take the max
    tot = red.sum(axis=0)
    for q in (0, 1, 2, 3, 4):
        assert tot[q] == pytest.approx(red_ref[0, q], rel=1e-12, abs=1e-12)
    assert red[:, 6].max() == red_ref[0, 6]
    assert red[:, 7].sum() == 0


def test_single_slab_is_the_periodic_grid():
    """One run with ACM_BC_HALO z faces exchanges with itself: the periodic
    grid again."""
    shape = (16, 20, 40)
    state = _fields(shape, seed=7)
    kw = dict(nu=0.03, precision=acm.FP32_DEV)
    ref, _ = _run(acm.make_params(shape, **kw), state, 25, (16,))
    got, _ = _run(acm.subdomain_params(shape, (16,), **kw), state, 25, (16,))
    for k in range(4):
        assert np.array_equal(got[k], ref[k])
