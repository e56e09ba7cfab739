"""Pins of the FP64 closure-network oracle (oracle/conv_ref.py) to facts that
do not come from the oracle: SciPy's periodic 2D correlation, the identity
kernel, central finite differences of the loss, and bfloat16 bit patterns."""
import numpy as np
import pytest

from oracle import conv_ref as cr


def test_conv_matches_scipy_periodic_correlation():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 9, 11))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cr.conv3x3(x, W, b)
    for co in range(4):
        ref = b[co] + sum(signal.correlate2d(x[ci], W[co, ci], mode="same", boundary="wrap")
                          for ci in range(3))
        assert np.abs(y[co] - ref).max() < 1e-12


def test_identity_and_shift_kernels():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 6, 7))
    W = np.zeros((2, 2, 3, 3))
    W[0, 0, 1, 1] = 1.0          # identity on channel 0
    W[1, 1, 1, 2] = 1.0          # y[1](i, j) = x[1](i, j + 1)
    y = cr.conv3x3(x, W, np.zeros(2))
    assert np.array_equal(y[0], x[0])
    assert np.array_equal(y[1], np.roll(x[1], -1, axis=1))


def test_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    params = cr.init_params(3, scale_out=0.5)
    x = rng.standard_normal((3, 6, 5))
    target = rng.standard_normal((3, 6, 5))
    loss, grads = cr.loss_and_grads(params, x, target)
    flat = cr.pack(params)
    gflat = cr.pack(grads)
    h = 1e-6
    idx = rng.choice(flat.size, 40, replace=False)
    for k in idx:
        fp = flat.copy()
        fp[k] += h
        fm = flat.copy()
        fm[k] -= h
        lp, _ = cr.loss_and_grads(cr.unpack(fp), x, target)
        lm, _ = cr.loss_and_grads(cr.unpack(fm), x, target)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[k]) < 1e-6 * max(1.0, abs(fd)), (k, fd, gflat[k])


def test_input_gradient_by_finite_differences():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 5, 6))
    W = rng.standard_normal((2, 3, 3, 3))
    dy = rng.standard_normal((2, 5, 6))
    dx, _, db = cr.conv3x3_grad(x, W, dy)
    h = 1e-6
    for _ in range(15):
        c, i, j = rng.integers(3), rng.integers(5), rng.integers(6)
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = ((dy * cr.conv3x3(xp, W, np.zeros(2))).sum() -
              (dy * cr.conv3x3(xm, W, np.zeros(2))).sum()) / (2 * h)
        assert abs(fd - dx[c, i, j]) < 1e-7
    assert np.allclose(db, dy.sum(axis=(1, 2)))


def test_bf16_rounding_bit_patterns():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties to even -> 1
    assert cr.to_bf16(1.0 + 2.0 ** -8) == 1.0
    assert cr.to_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert cr.to_bf16(3.140625) == 3.140625          # exactly representable
    assert cr.to_bf16(-2.0 ** -130) == -2.0 ** -130   # subnormal-range power of two
    x = np.random.default_rng(5).standard_normal(1000)
    r = cr.to_bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 + 1e-300)


def test_adam_first_step_is_signed_lr():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = cr.adam_update(p, g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-7)
