"""Multi-rank bookkeeping of the benchmark: every rank advances its own
independent replica of the workload (no data exchange between ranks); the job
time is the maximum over ranks and the throughput counts the node updates of
all ranks.  Only this timing reduction is collective."""
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
