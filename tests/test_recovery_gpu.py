"""Checkpoint/resume and failure reporting, all through the C ABI.

* Checkpoint/resume: 2n steps in one go equal n steps, a read-back of the
  fields (the checkpoint), a fresh handle restored from it, and n more steps:
  bit for bit with FP32 storage, to rounding with FP64 storage (2D single-
  and two-phase with walls, 3D): the state is exactly the stored fields,
  nothing hidden.
* Fault injection on the host: a non-finite value in the initial state is
  reported as ACM_EUNSTABLE by the next synchronising call, further steps
  are refused, and a clean set_fields clears the error; a handle survives.
* Allocation failure: a grid larger than the device is refused with
  ACM_ENOMEM on its first allocation, and later handles step normally (the
  failed call does not linger as the runtime's last error)."""
import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build
from test_parity_gpu import _smooth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    acm.load()


CASES = [
    ((48, 80), dict(nu=0.03)),
    ((40, 40), dict(nu=0.1, two_phase=True, sigma=1e-2, W=4.0, M=0.3, bc=[1, 1, 1, 1, 0, 0],
                    theta_deg=70.0)),
    ((20, 24, 40), dict(nu=0.04)),
]


def _state(shape, kw):
    rng = np.random.default_rng(31)
    st = [1 + 0.003 * _smooth(rng, shape)] + [0.02 * _smooth(rng, shape) for _ in shape]
    if kw.get("two_phase"):
        ny, nx = shape
        X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
        st.append(-np.tanh(2 * (np.hypot(X - 15.0, Y - 12.0) - 9.0) / 4.0))
        for a in st[1:3]:
            a[0, :] = a[-1, :] = 0.0
            a[:, 0] = a[:, -1] = 0.0
    return st


def _args(shape, st):
    if len(shape) == 3:
        return st[:4]
    return st[:3] + [None] + ([st[3]] if len(st) > 3 else [None])


@pytest.mark.parametrize("prec", [acm.FP64, acm.FP32_DEV])
@pytest.mark.parametrize("shape,kw", CASES)
def test_checkpoint_resume_bitwise(shape, kw, prec):
    st = _state(shape, kw)
    p = acm.make_params(shape, precision=prec, **kw)
    n = 37
    with acm.Solver(p) as s:
        s.set_fields(*_args(shape, st))
        s.step(2 * n)
        straight = s.fields()
    with acm.Solver(p) as s:
        s.set_fields(*_args(shape, st))
        s.step(n)
        ckpt = s.fields()
    with acm.Solver(p) as s:  # a new handle restored from the checkpoint
        s.set_fields(*_args(shape, [x for x in ckpt if x is not None]))
        s.step(n)
        resumed = s.fields()
    for a, b in zip(straight, resumed):
        if a is None:
            continue
        if prec == acm.FP32_DEV:
            assert np.array_equal(a, b)
        else:
            # the ABI exchanges absolute rho; in FP64 storage rho - rho0
            # comes back to within one ulp of rho, so the resumed run agrees
            # to rounding instead of bit for bit
            assert np.abs(a - b).max() <= 1e-14 * max(1.0, np.abs(a).max())


@pytest.mark.parametrize("shape", [(32, 48), (12, 16, 32)])
def test_nan_in_initial_state_is_reported_and_cleared(shape):
    st = [np.ones(shape)] + [np.zeros(shape) for _ in shape]
    st[1][tuple(s // 2 for s in shape)] = np.nan
    with acm.Solver(acm.make_params(shape, nu=0.05, precision=acm.FP32_DEV)) as s:
        s.set_fields(*st)
        s.step(3)
        with pytest.raises(acm.AcmError) as e:
            s.sync()
        assert e.value.status == acm.EUNSTABLE
        with pytest.raises(acm.AcmError):
            s.step(1)
        st[1][:] = 0.0
        s.set_fields(*st)
        s.step(5)
        s.sync()
        assert np.isfinite(s.fields()[1]).all()


def test_allocation_failure_leaves_the_context_usable():
    """A grid larger than the whole device (a periodic 4000^3 FP64 box: one
    field pool alone is about 514 GB) fails on its first allocation, before
    anything is held, with ACM_ENOMEM; the failed allocation does not linger
    as the runtime's last error, so handles created afterwards step and
    synchronise normally (and agree with each other bit for bit)."""
    with pytest.raises(acm.AcmError) as e:
        acm.Solver(acm.make_params((4000, 4000, 4000)))
    assert e.value.status in (acm.ENOMEM, acm.ECUDA)
    assert "cudaMalloc" in str(e.value)
    shape, kw = (12, 16, 32), dict(nu=0.04)
    st = _state(shape, kw)
    out = []
    for _ in range(2):
        with acm.Solver(acm.make_params(shape, **kw)) as s:
            s.set_fields(*st)
            s.step(10)
            s.sync()
            out.append(s.fields())
    for a, b in zip(out[0], out[1]):
        if a is not None:
            assert np.isfinite(a).all()
            assert np.array_equal(a, b)
