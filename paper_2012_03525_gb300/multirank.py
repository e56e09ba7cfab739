"""Multi-rank bookkeeping.  The benchmark's ranks advance independent
replicas of the workload (no data exchange between ranks); the job time is
the maximum over ranks and the throughput counts the node updates of all
ranks.  ``halo_exchange_z`` is the point-to-point exchange of a z-slab
decomposition of one grid over ranks."""
from __future__ import annotations


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank float over the process group (identity when
    ``dist`` is None or the group has one rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(nodes_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job lattice updates per second (GLUPS) of `world` replicas that
    each advanced `nodes_per_rank` nodes by `steps` steps within `seconds`."""
    return nodes_per_rank * steps * world / seconds / 1e9


def halo_exchange_z(fields, dist, ghost: int = 2) -> None:
    """Halo exchange of a z-slab decomposition over a process group: rank r
    holds planes of one periodic grid with ``ghost`` ghost planes beyond
    each z face (array axis 0), rank r+1 (mod world) the next slab above.
    Sends the top ``ghost`` interior planes of every field up and the bottom
    ones down, and fills the ghost planes from the neighbours -- the exchange
    step the library's sub-domain batches perform on one GPU with a
    halo-copy kernel.  ``fields`` are contiguous tensors [nz + 2 ghost][...];
    updated in place.  Point-to-point only (isend/irecv), so it runs on gloo
    (CPU tensors) as on NCCL."""
    rank, world = dist.get_rank(), dist.get_world_size()
    up, down = (rank + 1) % world, (rank - 1) % world
    g = ghost
    reqs, recv = [], []
    for k, f in enumerate(fields):
        top = f[-2 * g:-g].contiguous()      # last interior planes -> upper neighbour
        bottom = f[g:2 * g].contiguous()     # first interior planes -> lower neighbour
        lo = f.new_empty(f[:g].shape)
        hi = f.new_empty(f[-g:].shape)
        reqs.append(dist.isend(top, up, tag=2 * k))
        reqs.append(dist.isend(bottom, down, tag=2 * k + 1))
        reqs.append(dist.irecv(lo, down, tag=2 * k))
        reqs.append(dist.irecv(hi, up, tag=2 * k + 1))
        recv.append((f, lo, hi))
    for r in reqs:
        r.wait()
    for f, lo, hi in recv:
        f[:g] = lo
        f[-g:] = hi
