"""The benchmark's multi-rank path on CPU: two gloo ranks (127.0.0.1), each
reporting its own time; the job time is the maximum and the throughput counts
both replicas."""
import os

import pytest

from paper_2012_03525_gb300 import multirank


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = 1.0 + rank  # rank 1 is the slow one
    t = multirank.max_over_ranks(secs, dist)
    dist.barrier()
    q.put((rank, t, multirank.job_throughput(1000, 10, world, t)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, glups in out:
        assert t == 2.0
        assert glups == pytest.approx(1000 * 10 * 2 / 2.0 / 1e9)


def test_single_rank_is_identity():
    assert multirank.max_over_ranks(3.5, None) == 3.5
    assert multirank.job_throughput(10, 5, 1, 2.0) == 25 / 1e9
