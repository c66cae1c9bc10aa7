"""Host-side work split for one process per GPU.

The systems of a batched step are independent, so N GPUs share a batch by
taking disjoint sets of systems: no collective touches the data path, and
only the step time is reduced (the maximum over ranks).  The split balances
the history-slice work, which dominates a step: a system of M orbitals at
row n costs 8 M^3 (n+1)(3n+2) flops per slice (Eq. KBE2 over the 2n+1
required output blocks).  Systems are dealt largest first to the least
loaded rank (longest-processing-time rule, within 4/3 of the best split).
"""


def slice_cost(M, n):
    """Flops of one history slice of row n for M orbitals."""
    return 8.0 * M ** 3 * (n + 1) * (3 * n + 2)


def shard_systems(costs, world):
    """Indices of the systems each of ``world`` ranks takes, as a list of
    sorted lists; deterministic (ties by index), so every rank computes the
    same split without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    shards = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        shards[r].append(i)
        load[r] += float(costs[i])
    return [sorted(s) for s in shards]


def max_over_ranks(value):
    """The maximum of a float over the ranks of the default process group
    (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
