"""acm_reduce_mass_noalloc: the diagnostics for callers that cannot allocate
device memory (their device memory belongs to another runtime's allocator or
pool, or allocation is forbidden after start-up in a latency-bound loop).

The entry point keeps its scratch in fixed device arrays inside the library;
this file checks, through the C ABI, that two calls in a row give the same
answer as acm_reduce_mass on the same fields -- with the default block
count, one block, the full 4096 blocks the fixed scratch holds, more blocks
than the grid has nodes for (empty partials that pass 2 still combines), on
the legacy default stream and on a caller's stream, and on fields held as
absolute density or as the solver's deviation rho - rho0.  It sorts last so
that a run stopping at the first failure has already run every other test,
and it passes alone in a fresh process as well.
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


def _reference(shape, prec, rho0):
    rng = np.random.default_rng(21)
    dim = len(shape)
    st = [rho0 * (1 + 0.01 * _smooth(rng, shape))] + [0.03 * _smooth(rng, shape)
                                                      for _ in range(dim)]
    with acm.Solver(acm.make_params(shape, nu=0.05, precision=prec, rho0=rho0)) as s:
        s.set_fields(*st)
        s.step(2)
        prev = s.fields()
        s.step(1)
        cur = s.fields()
        ref = s.reduce()
    return cur, prev, ref


@pytest.mark.parametrize("shape,prec,rho0,deviation", [
    ((20, 24, 28), acm.FP64, 1.0, False), ((37, 50), acm.FP64, 1.0, False),
    ((18, 22, 26), acm.FP32_DEV, 1.0, False), ((18, 22, 26), acm.FP32_DEV, 2.5, True),
    ((37, 50), acm.FP64, 1.7, True)])
@pytest.mark.parametrize("blocks", [0, 1, 4096, "more"])
@pytest.mark.parametrize("own_stream", [False, True])
def test_noalloc_matches_reduce_mass_twice(torch_cuda, shape, prec, rho0, deviation, blocks,
                                           own_stream):
    torch = torch_cuda
    dim = len(shape)
    cur, prev, ref = _reference(shape, prec, rho0)
    n = int(np.prod(shape))
    if blocks == "more":
        blocks = (n + 255) // 256 + 37     # blocks beyond the grid: empty partials
    dt = torch.float64 if prec == acm.FP64 else torch.float32
    # deviation form: the array holds rho - rho0 (rounded to the storage type),
    # which is how the solver stores it; else absolute density
    r = cur[0] - rho0 if deviation else cur[0]
    dev = [torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)
           for x in (r, cur[1], cur[2], cur[3] if dim == 3 else cur[1])]
    pdev = [torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)
            for x in (prev[1], prev[2], prev[3] if dim == 3 else prev[1])]
    nz, ny, nx = shape if dim == 3 else (1,) + shape
    tol = 1e-12 if prec == acm.FP64 else 1e-6
    stream = torch.cuda.Stream() if own_stream else None
    handle = stream.cuda_stream if own_stream else 0
    if own_stream:
        stream.wait_stream(torch.cuda.current_stream())
    for _ in range(2):
        out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        if own_stream:
            stream.wait_stream(torch.cuda.current_stream())
        acm.reduce_mass_noalloc(dim, nx, ny, nz, prec, dev[0].data_ptr(), dev[1].data_ptr(),
                                dev[2].data_ptr(), dev[3].data_ptr() if dim == 3 else None,
                                (pdev[0].data_ptr(), pdev[1].data_ptr(),
                                 pdev[2].data_ptr() if dim == 3 else None),
                                blocks, out.data_ptr(), handle,
                                rho0=rho0 if deviation else 0.0)
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
