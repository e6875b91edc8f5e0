"""Host-side logic of the multi-GPU run: independent replicas.

The sampling path shards by samples with no exchange step, so N GPUs run N
independent replicas of the same step (weak scaling): each rank draws its own
batch from its own Philox key, and the only collectives are the barrier
around the timed region and a max over ranks of the elapsed time.  Nothing
here touches a GPU; the functions take a process group (NCCL in the bench,
gloo in the CPU tests).
"""
import torch


def replica_seed(rank: int, step: int) -> int:
    """Philox key of rank `rank` at step `step`: disjoint streams per rank
    (the rank sits in the key's upper 32 bits)."""
    if rank < 0 or rank >= 1 << 31:
        raise ValueError("rank out of range")
    return (rank << 32) + 1000 + step


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    x = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def whole_job_throughput(units_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    if seconds <= 0:
        raise ValueError("elapsed time must be positive")
    return units_per_rank * world * steps / seconds
