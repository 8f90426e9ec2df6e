"""Host-side bookkeeping for running independent problem replicas on N GPUs.

The solve shards by independent problems (RHS sets, frequencies, arrays):
each rank solves its own problems with no collective on the data path.  The
only communication is timing: a barrier around the timed region and the
maximum elapsed time over ranks, so throughput = all problems solved / the
slowest rank's time.
"""
import torch.distributed as dist


def world():
    """(world_size, rank) of the current process group, or (1, 0)."""
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def shard(items, rank, world_size):
    """Round-robin share of a list of independent problems for this rank."""
    return [x for i, x in enumerate(items) if i % world_size == rank]


def max_over_ranks(value, device="cpu"):
    """Maximum of a float over all ranks (the slowest replica's time)."""
    import torch
    w, _ = world()
    if w == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank, elapsed_s, device="cpu"):
    """Whole-job throughput: units solved on all ranks / max elapsed time."""
    import torch
    w, _ = world()
    total = float(units_per_rank)
    if w > 1:
        t = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total = float(t.item())
    return total / max_over_ranks(elapsed_s, device)
