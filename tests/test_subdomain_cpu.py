"""Slab decomposition of one periodic 3D grid over two gloo ranks (CPU): each
rank advances its z-slab with the NumPy oracle on the slab plus two ghost
planes per face, exchanging the ghost planes before every step
(``multirank.halo_exchange_z``).  The gathered result equals the unsplit
oracle run bit for bit: the scheme's stencil reaches two planes (one through
the fluxes and Laplacians of Eq. 2.11, one more through Delta rho of its
density-gradient SAT), so two ghost planes per face are exactly enough."""
import os

import numpy as np
import pytest

from paper_2012_03525_gb300 import multirank
from paper_2012_03525_gb300 import workloads as wl

SHAPE = (12, 10, 8)   # nz, ny, nx
SPLIT = (5, 7)
STEPS = 6
NU = 0.05
U0 = 0.08


def _fields():
    # anisotropic periodic box: a TGV-like field with a z dependence
    nz, ny, nx = SHAPE
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky, kz = 2 * np.pi / nx, 2 * np.pi / ny, 2 * np.pi / nz
    u = U0 * np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z)
    v = -U0 * np.cos(kx * x) * np.sin(ky * y) * np.cos(kz * z)
    w = 0.3 * U0 * np.sin(kz * z) * np.cos(kx * x)
    rho = 1.0 + 0.01 * np.cos(kx * x + 2 * kz * z)
    return [rho, u, v, w]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from oracle import ref_np
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    full = _fields()
    z0 = sum(SPLIT[:rank])
    n = SPLIT[rank]
    slab = [torch.zeros((n + 4,) + f.shape[1:], dtype=torch.float64) for f in full]
    for t, f in zip(slab, full):
        t[2:-2] = torch.from_numpy(f[z0:z0 + n])
    for _ in range(STEPS):
        multirank.halo_exchange_z(slab, dist)
        rho, vel, _ = ref_np.step(slab[0].numpy(), [s.numpy() for s in slab[1:]], nsteps=1,
                                  nu=NU)
        for t, a in zip(slab, [rho] + vel):
            t[2:-2] = torch.from_numpy(a[2:-2])
    q.put((rank, [t[2:-2].numpy().copy() for t in slab]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_slabs_equal_unsplit_oracle_bitwise():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    from oracle import ref_np
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = _fields()
    rho, vel, _ = ref_np.step(full[0], full[1:], nsteps=STEPS, nu=NU)
    ref = [rho] + vel
    for k in range(4):
        joined = np.concatenate([got[0][k], got[1][k]], axis=0)
        assert np.array_equal(joined, ref[k]), k


def test_ghost_depth_one_is_not_enough():
    """With only one ghost plane per face filled exactly (the outer one
    zeroed), rho, u and v of the slab still match the unsplit step -- their
    stencils reach one plane in z -- but w does not: its density-gradient SAT
    d_z(rho^{n+1} - rho^n) of Eq. 2.11 takes Delta rho one plane beyond the
    face, which needs the second ghost plane."""
    from oracle import ref_np
    full = _fields()
    rho, vel, _ = ref_np.step(full[0], full[1:], nsteps=1, nu=NU)
    n = SPLIT[0]
    pad = [np.concatenate([f[-2:], f[:n], f[n:n + 2]], axis=0) for f in full]
    for f in pad:
        f[0] = 0.0       # the outer ghost plane below is missing
        f[-1] = 0.0      # and the one above
    r1, v1, _ = ref_np.step(pad[0], pad[1:], nsteps=1, nu=NU)
    assert np.array_equal(r1[2:-2], rho[:n])
    assert np.array_equal(v1[0][2:-2], vel[0][:n])
    assert np.array_equal(v1[1][2:-2], vel[1][:n])
    assert not np.array_equal(v1[2][2], vel[2][0])
    assert not np.array_equal(v1[2][-3], vel[2][n - 1])
    assert np.array_equal(v1[2][3:-3], vel[2][1:n - 1])
