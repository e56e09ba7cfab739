"""GPU parity of the learned closure's tensor-core kernels against the FP64
oracle (oracle/conv_ref.py), run through the C ABI.

The oracle receives the same quantised operands the kernels use (inputs and
weights rounded to bfloat16, hidden activations and activation gradients
rounded where the kernels store them), so the remaining differences are the
FP32 accumulation order and rare bfloat16 rounding flips of stored values.
Tolerances: network output relative L2 <= 2e-3, weight gradients <= 2e-2
per layer, loss <= 1e-5 relative.
"""
import numpy as np
import pytest

from oracle import conv_ref as cr
from paper_2012_03525_gb300 import acm, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("needs a GPU")
    build.build()
    acm.load()
    return t


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


def quantised_params(seed, scale_out):
    params = cr.init_params(seed, scale_out=scale_out)
    rng = np.random.default_rng(seed + 100)
    out = []
    for W, b in params:
        b = rng.standard_normal(b.shape) * 0.05
        out.append((cr.to_bf16(W), np.float32(b).astype(np.float64)))
    return out


def test_forward_matches_oracle(torch):
    B, H, W = 2, 32, 48
    rng = np.random.default_rng(0)
    x = cr.to_bf16(rng.standard_normal((B, 3, H, W)))
    params = quantised_params(1, 0.5)
    with acm.Closure(W, H, B) as c:
        c.set_weights(cr.pack(params).astype(np.float32))
        xd = torch.from_numpy(x.astype(np.float32)).cuda()
        nd = torch.zeros_like(xd)
        c.forward(xd.data_ptr(), nd.data_ptr())
        torch.cuda.synchronize()
        got = nd.cpu().numpy().astype(np.float64)
    for b in range(B):
        ref, _ = cr.forward(params, x[b], bf16_activations=True)
        assert rel(got[b], ref) < 2e-3, rel(got[b], ref)


def test_loss_and_gradients_match_oracle(torch):
    B, H, W = 2, 16, 32
    rng = np.random.default_rng(2)
    x = cr.to_bf16(rng.standard_normal((B, 3, H, W)))
    target = rng.standard_normal((B, 3, H, W))
    params = quantised_params(3, 0.5)
    with acm.Closure(W, H, B) as c:
        c.set_weights(cr.pack(params).astype(np.float32))
        xd = torch.from_numpy(x.astype(np.float32)).cuda()
        td = torch.from_numpy(target.astype(np.float32)).cuda()
        loss, g = c.loss_grad(xd.data_ptr(), td.data_ptr())
    # the batch loss is the mean over all images: sum the per-image oracle
    # gradients scaled by 1/B (each image's loss is a mean over its elements)
    ref_loss = 0.0
    ref_g = np.zeros(cr.n_params())
    for b in range(B):
        l, gr = cr.loss_and_grads(params, x[b], target[b].astype(np.float32).astype(np.float64),
                                  bf16_activations=True, bf16_grads=False)
        ref_loss += l / B
        ref_g += cr.pack(gr) / B
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    k = 0
    for l in range(3):
        nW = cr.CH[l + 1] * cr.CH[l] * 9
        nb = cr.CH[l + 1]
        assert rel(g[k:k + nW], ref_g[k:k + nW]) < 2e-2, (l, rel(g[k:k + nW], ref_g[k:k + nW]))
        assert rel(g[k + nW:k + nW + nb], ref_g[k + nW:k + nW + nb]) < 2e-2
        k += nW + nb


def test_adam_step_and_training_reduces_loss(torch):
    """A student closure learns a fixed random teacher closure's correction;
    the first Adam step moves every weight by lr * sign(g)."""
    B, H, W = 4, 32, 32
    rng = np.random.default_rng(4)
    teacher = quantised_params(5, 0.3)
    xs, ts = [], []
    for _ in range(B):
        x = cr.to_bf16(rng.standard_normal((3, H, W)))
        out, _ = cr.forward(teacher, x)
        xs.append(x)
        ts.append(x + out)
    x = np.stack(xs).astype(np.float32)
    target = np.stack(ts).astype(np.float32)
    student = cr.pack(cr.init_params(6, scale_out=1e-2)).astype(np.float32)
    with acm.Closure(W, H, B) as c:
        c.set_weights(student)
        xd = torch.from_numpy(x).cuda()
        td = torch.from_numpy(target).cuda()
        loss0, g0 = c.loss_grad(xd.data_ptr(), td.data_ptr())
        lr = 1e-3
        c.train_step(xd.data_ptr(), td.data_ptr(), lr)
        w1 = c.get_weights()
        step = w1.astype(np.float64) - student
        big = np.abs(g0) > 1e-4  # eps = 1e-8 shrinks steps of tiny gradients
        assert np.allclose(step[big], -lr * np.sign(g0[big]), rtol=1e-3, atol=1e-6)
        losses = [c.train_step(xd.data_ptr(), td.data_ptr(), 3e-3) for _ in range(300)]
    assert losses[-1] < 0.2 * loss0, (loss0, losses[::50])


def test_apply_adds_bias_correction_to_solver_state(torch):
    """With zero weights and a bias b on the output layer the closure adds
    exactly b / scale to each field of every run."""
    n, B = 32, 2
    params = [acm.make_params((n, n), nu=0.05, precision=acm.FP32_DEV) for _ in range(B)]
    rng = np.random.default_rng(7)
    w = np.zeros(cr.n_params(), dtype=np.float32)
    bias = np.array([0.5, -0.25, 0.125], dtype=np.float32)
    w[-3:] = bias
    s_rho, s_u = 100.0, 20.0
    with acm.Solver(params) as s, acm.Closure(n, n, B) as c:
        states = []
        for r in range(B):
            st = [1 + 1e-3 * rng.standard_normal((n, n)), 0.01 * rng.standard_normal((n, n)),
                  0.01 * rng.standard_normal((n, n))]
            s.set_fields(*st, run=r)
            states.append(s.fields(run=r))
        c.set_scales(s_rho, s_u)
        c.set_weights(w)
        c.apply(s)
        for r in range(B):
            got = s.fields(run=r)
            assert np.allclose(got[0] - states[r][0], bias[0] / s_rho, atol=1e-6)
            assert np.allclose(got[1] - states[r][1], bias[1] / s_u, atol=1e-6)
            assert np.allclose(got[2] - states[r][2], bias[2] / s_u, atol=1e-6)


def test_input_noise_is_seeded_and_off_by_default(torch):
    """acm_closure_set_input_noise: sigma = 0 leaves the loss unchanged; a
    given seed reproduces the same noisy loss (counter-based normals); the
    noise raises the loss of a closure that fits the clean data."""
    B, H, W = 2, 16, 32
    rng = np.random.default_rng(6)
    x = cr.to_bf16(rng.standard_normal((B, 3, H, W)))
    target = rng.standard_normal((B, 3, H, W))
    params = quantised_params(8, 0.5)
    with acm.Closure(W, H, B) as c:
        c.set_weights(cr.pack(params).astype(np.float32))
        xd = torch.from_numpy(x.astype(np.float32)).cuda()
        td = torch.from_numpy(target.astype(np.float32)).cuda()
        l0, _ = c.loss_grad(xd.data_ptr(), td.data_ptr())
        c.set_input_noise(0.0, 3)
        l1, _ = c.loss_grad(xd.data_ptr(), td.data_ptr())
        c.set_input_noise(0.5, 3)
        la, _ = c.loss_grad(xd.data_ptr(), td.data_ptr())
        c.set_input_noise(0.5, 3)   # resets the call counter
        lb, _ = c.loss_grad(xd.data_ptr(), td.data_ptr())
        c.set_input_noise(0.5, 4)
        lc, _ = c.loss_grad(xd.data_ptr(), td.data_ptr())
    assert l1 == l0
    assert la == lb and la != l0 and lc != la


def test_pushforward_samples_restart_every_r_windows(torch):
    """Data aggregation with restarts (closure.generate, reset_every = r):
    the windows that start from the filtered fine state give exactly the
    one-window samples; the windows in between start from the corrected
    state, so they differ; targets are the filtered fine states throughout."""
    from paper_2012_03525_gb300 import closure as cl
    setup = cl.Setup(n_fine=128, factor=4, window=4)
    seeds, B = [0, 1], 2
    X1, Y1 = cl.generate(setup, seeds, 4, torch, B, reset=True)
    clo = acm.Closure(setup.n_coarse, setup.n_coarse, B)
    clo.set_scales(*setup.scales())
    w = cl.he_init(0, scale_out=1.0)  # a correction large enough to matter
    clo.set_weights(w)
    X2, Y2 = cl.generate(setup, seeds, 4, torch, B, model=clo, reset_every=2)
    torch.cuda.synchronize()
    assert X2.shape == X1.shape
    assert torch.equal(Y1, Y2)
    for k in (0, 2):
        assert torch.equal(X1[k], X2[k])
    for k in (1, 3):
        assert not torch.equal(X1[k], X2[k])
    clo.close()
