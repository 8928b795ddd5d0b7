"""Replica parallelism over ranks (one process per GPU).

The hot path has no exchange step: on N GPUs every rank advances its own,
independently seeded box (weak scaling).  The only communication is a
barrier around timed regions and the maximum of the ranks' times; these
helpers hold that host logic so that it can be tested with the gloo backend
on CPU.
"""
import os

import torch


def rank_info(env=None):
    """(rank, world size, local rank) from the launcher's environment."""
    env = os.environ if env is None else env
    return int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")), int(env.get("LOCAL_RANK", "0"))


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank's workload: distinct per rank, rank 0 keeps the base seed."""
    return base + rank


def shard(n_units: int, rank: int, world: int):
    """Contiguous block [lo, hi) of n_units independent units for rank; the
    blocks of all ranks partition the units and differ in size by at most one."""
    per, extra = divmod(n_units, world)
    lo = rank * per + min(rank, extra)
    return lo, lo + per + (1 if rank < extra else 0)


def _initialized():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized()


def barrier(cuda: bool = True):
    """All ranks reach this point (and, with cuda, their streams are drained)."""
    if _initialized():
        import torch.distributed as dist
        dist.barrier()
    if cuda and torch.cuda.is_available():
        torch.cuda.synchronize()


def max_over_ranks(value: float, device=None) -> float:
    """The largest of the ranks' values (the job's time is the slowest rank's)."""
    if not _initialized():
        return float(value)
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
