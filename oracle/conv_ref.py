"""FP64 reference of the learned closure's network (test infrastructure only).

The closure is a 3-layer stack of 3x3 convolutions on a periodic 2D grid,
channels 3 -> 32 -> 32 -> 3, ReLU after the first two layers, whose output is
added to the coarse-grid state (rho', u, v) after a solver step.  Everything
here is plain NumPy in float64 written from the definition of a 2D
cross-correlation with periodic wrap:

    y[co, i, j] = b[co] + sum_{ci, di, dj} W[co, ci, di+1, dj+1] x[ci, i+di, j+dj]

(di, dj in {-1, 0, 1}, indices modulo the grid), its gradients by the chain
rule, and the mean-squared-error loss.  ``to_bf16`` rounds to bfloat16
(round to nearest even) so a test can give the oracle the same quantised
operands the tensor-core kernels use; ``bf16_activations=True`` rounds the
stored hidden activations at the same points the kernels store them.
"""
from __future__ import annotations

import numpy as np

CH = (3, 32, 32, 3)


def to_bf16(x):
    """Round float values to the nearest bfloat16 (ties to even), returned as
    float64.  bfloat16 keeps the top 16 bits of the IEEE float32 pattern."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = (bits + 0x7FFF + lsb) >> 16
    out = (rounded << 16).astype(np.uint32).view(np.float32)
    return out.astype(np.float64)


def shift(x, di, dj):
    """x[..., i + di, j + dj] with periodic wrap."""
    return np.roll(np.roll(x, -di, axis=-2), -dj, axis=-1)


def conv3x3(x, W, b):
    """x: (Cin, H, W); W: (Cout, Cin, 3, 3); b: (Cout,) -> (Cout, H, W)."""
    cout = W.shape[0]
    y = np.zeros((cout,) + x.shape[1:])
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            xs = shift(x, di, dj)
            y += np.einsum("oc,chw->ohw", W[:, :, di + 1, dj + 1], xs)
    return y + b[:, None, None]


def conv3x3_grad(x, W, dy):
    """Gradients of sum(dy * conv3x3(x, W, b)) w.r.t. x, W and b."""
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            xs = shift(x, di, dj)
            dW[:, :, di + 1, dj + 1] = np.einsum("ohw,chw->oc", dy, xs)
            # y at (i, j) used x at (i + di, j + dj): move dy back by (di, dj)
            dx += shift(np.einsum("oc,ohw->chw", W[:, :, di + 1, dj + 1], dy), -di, -dj)
    return dx, dW, dy.sum(axis=(1, 2))


def init_params(seed=0, scale_out=1e-2):
    """He-style initial weights (FP64); the last layer is scaled down so the
    untrained closure starts close to the identity correction (zero)."""
    rng = np.random.default_rng(seed)
    params = []
    for l in range(3):
        cin, cout = CH[l], CH[l + 1]
        std = np.sqrt(2.0 / (9 * cin))
        if l == 2:
            std *= scale_out
        params.append((rng.standard_normal((cout, cin, 3, 3)) * std, np.zeros(cout)))
    return params


def forward(params, x, bf16_activations=False):
    """Returns the correction (3, H, W) and the hidden activations."""
    q = to_bf16 if bf16_activations else (lambda a: a)
    h1 = q(np.maximum(conv3x3(x, *params[0]), 0.0))
    h2 = q(np.maximum(conv3x3(h1, *params[1]), 0.0))
    out = conv3x3(h2, *params[2])
    return out, (h1, h2)


def loss_and_grads(params, x, target, bf16_activations=False, bf16_grads=False):
    """MSE loss mean((x + net(x) - target)^2) over all elements and the
    gradients of every weight and bias (x is not differentiated).
    ``bf16_grads`` rounds the stored activation gradients (d loss / d out and
    the masked hidden-layer gradients) to bfloat16 where the kernels store
    them."""
    qg = to_bf16 if bf16_grads else (lambda a: a)
    out, (h1, h2) = forward(params, x, bf16_activations)
    r = x + out - target
    n = r.size
    loss = float((r * r).sum() / n)
    d3 = qg(2.0 * r / n)
    dh2, dW3, db3 = conv3x3_grad(h2, params[2][0], d3)
    dh2 = qg(dh2 * (h2 > 0))
    dh1, dW2, db2 = conv3x3_grad(h1, params[1][0], dh2)
    dh1 = qg(dh1 * (h1 > 0))
    _, dW1, db1 = conv3x3_grad(x, params[0][0], dh1)
    return loss, [(dW1, db1), (dW2, db2), (dW3, db3)]


def pack(params):
    """Flatten to the library's weight vector order: per layer W[co][ci][3][3]
    then b[co]."""
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unpack(vec):
    params, k = [], 0
    for l in range(3):
        cin, cout = CH[l], CH[l + 1]
        nW = cout * cin * 9
        W = np.asarray(vec[k:k + nW], dtype=np.float64).reshape(cout, cin, 3, 3)
        k += nW
        b = np.asarray(vec[k:k + cout], dtype=np.float64)
        k += cout
        params.append((W, b))
    return params


def n_params():
    return sum(CH[l + 1] * CH[l] * 9 + CH[l + 1] for l in range(3))


def adam_update(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) on flat arrays; returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
