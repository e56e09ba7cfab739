"""The native autotuner on every kind of handle: it times trial steps on a
copy of the state, leaves the fields untouched, and the launch shape it picks
changes no bit of the result (the kernels' arithmetic does not depend on the
tile height, z-chunking or persistent-CTA count)."""
import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build
from test_parity_gpu import _smooth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    acm.load()


def _case(kind):
    rng = np.random.default_rng(21)
    if kind == "mames":
        shape = (48, 70)
        st = [1 + 0.002 * _smooth(rng, shape)] + [0.03 * _smooth(rng, shape) for _ in range(2)]
        return [acm.make_params(shape, nu=0.04, scheme=acm.SCHEME_MAMES,
                                precision=acm.FP32_DEV)], [st]
    if kind == "twophase3d":
        shape = (16, 20, 36)
        Z, Y, X = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
        phi = -np.tanh(2.0 * (np.sqrt((X - 17.5) ** 2 + (Y - 9.5) ** 2 + Z ** 2) - 7.0) / 4.0)
        z = np.zeros(shape)
        st = [np.ones(shape), 1e-3 * _smooth(rng, shape), z, z.copy(), phi]
        st[1][0] = 0.0
        st[1][-1] = 0.0
        return [acm.make_params(shape, dt=0.5, nu=0.1, bc=[0, 0, 0, 0, 1, 1], two_phase=True,
                                sigma=1e-2, W=4.0, M=0.5, theta_deg=70.0)], [st]
    # sub-domains: a 3D periodic grid as three z-slabs
    shape = (30, 24, 40)
    full = [1 + 0.005 * _smooth(rng, shape)] + [0.03 * _smooth(rng, shape) for _ in range(3)]
    parts = (9, 11, 10)
    params = acm.subdomain_params(shape, parts, nu=0.03, precision=acm.FP32_DEV)
    sts, z0 = [], 0
    for n in parts:
        sts.append([f[z0:z0 + n].copy() for f in full])
        z0 += n
    return params, sts


@pytest.mark.parametrize("kind", ["mames", "twophase3d", "subdomains"])
def test_autotune_every_handle_kind(kind):
    params, states = _case(kind)
    arg = params if len(params) > 1 else params[0]
    out = []
    for tune in (False, True):
        with acm.Solver(arg) as s:
            for r, st in enumerate(states):
                s.set_fields(*st, run=r)
            before = [s.fields(run=r) for r in range(len(states))]
            if tune:
                assert s.autotune(3) > 0
                after = [s.fields(run=r) for r in range(len(states))]
                for fa, fb in zip(before, after):
                    for a, b in zip(fa, fb):
                        if a is not None:
                            assert np.array_equal(a, b)
            s.step(30)
            out.append([s.fields(run=r) for r in range(len(states))])
    for fa, fb in zip(out[0], out[1]):
        for a, b in zip(fa, fb):
            if a is not None:
                assert np.array_equal(a, b)
