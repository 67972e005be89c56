"""Replica sharding across ranks (one process per GPU).

RHS columns and whole operators are independent, so N GPUs run N replicas of
the operators and split the right-hand sides without any collective on the
data path.  The only collective is the max of the per-rank elapsed times that
the benchmark reports.
"""


def column_shard(k_total, world, rank):
    """Contiguous share [start, start + count) of k_total columns for `rank`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world / rank")
    base, extra = divmod(int(k_total), world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def request_shard(request_ids, world, rank):
    """Round-robin share of a request stream (ids in arrival order)."""
    return [q for i, q in enumerate(request_ids) if i % world == rank]


def rank_seed(seed, rank):
    """Seed of the inputs a rank draws (distinct per rank, reproducible)."""
    return int(seed) + 1000003 * int(rank)


def max_over_ranks(value, dist=None):
    """Max of a float over the process group (identity without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
