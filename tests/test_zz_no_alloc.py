"""acm_reduce_mass_noalloc: the diagnostics for callers that cannot allocate
device memory (their device memory belongs to another runtime's allocator or
pool, or allocation is forbidden after start-up in a latency-bound loop).

The entry point keeps its scratch in fixed device arrays inside the library;
this file checks, through the C ABI, that two calls in a row give the same
answer as acm_reduce_mass on the same fields.  It sorts last so that a run
stopping at the first failure has already run every other test, and it
passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_2012_03525_gb300 import acm, build

pytestmark = pytest.mark.gpu


def _smooth(rng, shape, kmax2=6):
    f = rng.standard_normal(shape)
    F = np.fft.fftn(f)
    ks = np.meshgrid(*[np.fft.fftfreq(n) * n for n in shape], indexing="ij")
    F[sum(k * k for k in ks) > kmax2] = 0
    return np.ascontiguousarray(np.real(np.fft.ifftn(F)))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    build.build()
    acm.load()
    return torch


@pytest.mark.parametrize("shape,prec", [((20, 24, 28), acm.FP64), ((37, 50), acm.FP64),
                                        ((18, 22, 26), acm.FP32_DEV)])
def test_noalloc_matches_reduce_mass_twice(torch_cuda, shape, prec):
    torch = torch_cuda
    rng = np.random.default_rng(21)
    dim = len(shape)
    st = [1 + 0.01 * _smooth(rng, shape)] + [0.03 * _smooth(rng, shape) for _ in range(dim)]
    with acm.Solver(acm.make_params(shape, nu=0.05, precision=prec)) as s:
        s.set_fields(*st)
        s.step(2)
        prev = s.fields()
        s.step(1)
        cur = s.fields()
        ref = s.reduce()

    dt = torch.float64 if prec == acm.FP64 else torch.float32
    dev = [torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)
           for x in (cur[0], cur[1], cur[2], cur[3] if dim == 3 else cur[1])]
    pdev = [torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)
            for x in (prev[1], prev[2], prev[3] if dim == 3 else prev[1])]
    nz, ny, nx = shape if dim == 3 else (1,) + shape
    tol = 1e-12 if prec == acm.FP64 else 1e-6
    for _ in range(2):
        out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        acm.reduce_mass_noalloc(dim, nx, ny, nz, prec, dev[0].data_ptr(), dev[1].data_ptr(),
                                dev[2].data_ptr(), dev[3].data_ptr() if dim == 3 else None,
                                (pdev[0].data_ptr(), pdev[1].data_ptr(),
                                 pdev[2].data_ptr() if dim == 3 else None),
                                0, out.data_ptr(), 0)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = abs(ref[0])
        for q in (0, 1, 2, 3, 4):
            assert got[q] == pytest.approx(ref[q], rel=tol, abs=tol * scale), (q, got, ref)
        for q in (5, 6):
            assert got[q] == pytest.approx(ref[q], rel=tol)
        assert got[7] == 0.0


def test_noalloc_rejects_too_many_blocks(torch_cuda):
    torch = torch_cuda
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(acm.AcmError) as e:
        acm.reduce_mass_noalloc(2, 8, 8, 1, acm.FP64, x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                None, None, 5000, out.data_ptr(), 0)
    assert e.value.status == acm.EINVAL
    assert "4096" in str(e.value)
