"""Oracle parity on the persistent multi-item path of the 2D kernels.

The 2D step kernels (single-phase, two-phase and the MAMEs comparison
scheme) launch at most SMs x occupancy CTAs that walk a (run, tile) work
list; a CTA with more than one item stages the next item's tiles while it
computes the current one.  These tests force that path with few CTAs
(acm_set_tuning ACM_TUNE_BLOCKS = 1, 7, SMs) on grids of hundreds of tiles
and on a seeded subset of the batched-drop workload that includes its
largest grids, and compare every run with the FP64 oracle."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build
from paper_2012_03525_gb300 import workloads as wl
from test_parity_gpu import assert_parity, _flow, _smooth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sms():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    build.build()
    acm.load()
    return torch.cuda.get_device_properties(0).multi_processor_count


def _gpu(params, states, steps, blocks):
    with acm.Solver(params) as s:
        s.set_tuning(acm.TUNE_BLOCKS, blocks)
        s.set_tuning(acm.TUNE_LINE2D, 0)  # the tile kernel's persistent path
        for r, st in enumerate(states):
            s.set_fields(st[0], st[1], st[2], None, st[3] if len(st) > 3 else None, run=r)
        s.step(steps)
        return [list(s.fields(run=r)) for r in range(len(states))]


@pytest.fixture(scope="module")
def tgv512(oracle_lib):
    co = oracle_lib
    n, steps = 512, 40
    st = [x + 0 for x in wl.tgv2d(n, 0.05)]
    rng = np.random.default_rng(5)
    st[1] = st[1] + 0.01 * _smooth(rng, (n, n))
    ref = [x.copy() for x in st]
    co.step(co.make_params((n, n), nu=0.02), *ref, nsteps=steps)
    return st, ref, steps


@pytest.mark.parametrize("blocks_of", ["1", "7", "sms"])
@pytest.mark.parametrize("prec", [acm.FP64, acm.FP32_DEV])
def test_tgv512_persistent_ctas(sms, tgv512, blocks_of, prec):
    st, ref, steps = tgv512
    blocks = {"1": 1, "7": 7, "sms": sms}[blocks_of]
    got = _gpu([acm.make_params((512, 512), nu=0.02, precision=prec)], [st], steps, blocks)[0]
    if prec == acm.FP64:
        assert_parity(ref + [None, None], got)
    else:
        assert_parity(ref + [None, None], got, tol=2e-5, tol_rho=1e-4)


@pytest.mark.parametrize("blocks_of", ["7", "sms"])
def test_cavity_persistent_ctas(sms, oracle_lib, blocks_of):
    co = oracle_lib
    n, steps, lid = 384, 60, 0.1
    bc = [1, 1, 1, 2, 0, 0]
    st = list(wl.cavity2d(n, lid))
    ref = [x.copy() for x in st]
    co.step(co.make_params((n, n), nu=0.05, bc=bc, lid_u=(lid, 0, 0)), *ref, nsteps=steps)
    blocks = {"7": 7, "sms": sms}[blocks_of]
    got = _gpu([acm.make_params((n, n), nu=0.05, bc=bc, lid_u=(lid, 0, 0))], [st], steps,
               blocks)[0]
    assert_parity(ref + [None, None], got)


@pytest.mark.parametrize("blocks_of", ["1", "sms"])
def test_mames_persistent_ctas(sms, oracle_lib, blocks_of):
    co = oracle_lib
    n, steps = 320, 40
    st = list(wl.tgv2d(n, 0.04))
    ref = [x.copy() for x in st]
    co.step_mames(co.make_params((n, n), nu=0.03), *ref, nsteps=steps)
    blocks = {"1": 1, "sms": sms}[blocks_of]
    got = _gpu([acm.make_params((n, n), nu=0.03, scheme=acm.SCHEME_MAMES)], [st], steps,
               blocks)[0]
    assert_parity(ref + [None, None], got)


def _drop_subset(k=24):
    """A seeded subset of the 512-run batched-drop workload: the four largest
    grids and k - 4 others drawn with a fixed seed."""
    runs = wl.batch_drops()
    order = np.argsort([r.n for r in runs])
    pick = list(order[-4:]) + list(np.random.default_rng(77).choice(order[:-4], k - 4,
                                                                    replace=False))
    return [runs[i] for i in pick]


@pytest.fixture(scope="module")
def drops(oracle_lib):
    """Initial states (drop + a smooth flow, so every term acts from the
    first step) and the oracle after ``steps`` steps, one host thread per
    run (the oracle releases the interpreter lock)."""
    co = oracle_lib
    runs, steps = _drop_subset(), 30
    rng = np.random.default_rng(8)
    states = []
    for r in runs:
        rho, u, v, phi = wl.drop2d(r.n, r.radius, r.W, eps=r.eps)
        states.append([rho, u + _flow(rng, u.shape), v + _flow(rng, v.shape), phi])

    def one(i):
        r = runs[i]
        st = [x.copy() for x in states[i]]
        p = co.make_params((r.n, r.n), nu=r.nu, two_phase=True, sigma=r.sigma, W=r.W, M=r.M)
        co.step(p, st[0], st[1], st[2], None, st[3], nsteps=steps)
        return st

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(runs), os.cpu_count() or 1))) as ex:
        refs = list(ex.map(one, range(len(runs))))
    return runs, states, refs, steps


@pytest.mark.parametrize("blocks_of", ["7", "sms"])
def test_drop_batch_subset_persistent(sms, drops, blocks_of):
    """24 runs of the seeded drop batch (grids 64^2-512^2, its four largest
    included) in one handle: FP64 two-phase, every run equals its oracle
    run at 1e-12."""
    runs, states, refs, steps = drops
    assert max(r.n for r in runs) >= 500
    params = [acm.make_params((r.n, r.n), nu=r.nu, two_phase=True, sigma=r.sigma, W=r.W, M=r.M)
              for r in runs]
    blocks = {"7": 7, "sms": sms}[blocks_of]
    got = _gpu(params, states, steps, blocks)
    bad = []
    for i, (ref, g) in enumerate(zip(refs, got)):
        try:
            assert_parity([ref[0], ref[1], ref[2], None, ref[3]], g)
        except AssertionError as e:
            bad.append((i, runs[i].n, str(e)[:120]))
    assert not bad, bad


def test_drop_batch_laplace_law(sms):
    """The Laplace-law check of the batched-drop workload: the seeded subset
    as static drops (eps = 0, at rest), FP32 deviation storage as in the
    benchmark; after 400 steps the interface-weighted chemical potential of
    every run is within 5 % of sigma / (2 R_eff) (Section 2's mu; the Laplace
    law in 2D), computed on the device by acm_reduce_laplace."""
    runs = _drop_subset()
    params = [acm.make_params((r.n, r.n), nu=r.nu, two_phase=True, sigma=r.sigma, W=r.W, M=r.M,
                              precision=acm.FP32_DEV) for r in runs]
    with acm.Solver(params) as s:
        for i, r in enumerate(runs):
            st = wl.drop2d(r.n, r.radius, r.W)
            s.set_fields(st[0], st[1], st[2], None, st[3], run=i)
        s.step(400)
        lap = s.reduce_laplace()
    ratio = lap[:, 2] / lap[:, 6]
    assert np.all(np.abs(ratio - 1) < 0.05), ratio
    # the drop area is conserved by the Cahn-Hilliard step: R_eff stays R
    radii = np.array([r.radius for r in runs])
    assert np.all(np.abs(lap[:, 1] / radii - 1) < 0.02), lap[:, 1] / radii
