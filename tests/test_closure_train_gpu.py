"""End-to-end learned closure on a reduced set-up: training data from fine
FP64 runs of the scheme, training on the GPU with the library's kernels, and
the gain on held-out initial conditions: the corrected coarse run must be
closer to the filtered fine reference than the plain coarse run."""
import pytest

from paper_2012_03525_gb300 import acm, build
from paper_2012_03525_gb300 import closure as cl
from paper_2012_03525_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("needs a GPU")
    build.build()
    acm.load()
    return t


def test_restriction_of_uniform_and_scaled_fields(torch):
    """acm_restrict: block means with the lattice unit change (u / factor,
    rho' / factor^2) into a coarse handle and a normalised buffer."""
    import numpy as np
    n, f = 64, 4
    rng = np.random.default_rng(0)
    fine = acm.Solver([acm.make_params((n, n), nu=0.05)])
    rho = 1 + 1e-3 * rng.standard_normal((n, n))
    u, v = 0.01 * rng.standard_normal((n, n)), 0.01 * rng.standard_normal((n, n))
    fine.set_fields(rho, u, v)
    coarse = acm.Solver([acm.make_params((n // f, n // f), nu=0.05, precision=acm.FP32_DEV)])
    fine.restrict_to(coarse, f)
    got = coarse.fields()
    bm = lambda a: a.reshape(n // f, f, n // f, f).mean(axis=(1, 3))
    assert np.allclose(got[0] - 1, bm(rho - 1) / f ** 2, atol=1e-9)
    assert np.allclose(got[1], bm(u) / f, atol=1e-8)
    out = torch.empty((1, 3, n // f, n // f), device="cuda", dtype=torch.float32)
    fine.restrict_to(None, f, out_dev=out.data_ptr(), scales=(10.0, 3.0))
    o = out.cpu().numpy()[0]
    assert np.allclose(o[2], 3.0 * bm(v) / f, atol=1e-7)
    fine.close()
    coarse.close()


def test_trained_closure_reduces_one_window_error(torch):
    """Trained on windows restarted from filtered fine states of 16 training
    trajectories, the closure cuts the one-window velocity error on held-out
    initial conditions (measured: 0.136 -> 0.054 at 32^2 from 128^2)."""
    setup = cl.Setup(n_fine=128, factor=4, window=8, dt=0.02)
    batch = 4
    X, Y = cl.generate(setup, list(wl.TURB_TRAIN_SEEDS)[:16], windows=12, torch=torch,
                       batch=batch, reset=True)
    closure, losses = cl.train(setup, X, Y, torch, batch, epochs=20, lr=1e-3)
    assert losses[-1] < 0.3 * losses[0], losses
    res = cl.evaluate_windows(setup, closure, list(wl.TURB_TEST_SEEDS)[:batch], 6, torch, batch)
    assert res["closure"] < 0.7 * res["plain"], res
    closure.close()
