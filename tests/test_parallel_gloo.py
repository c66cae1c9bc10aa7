"""The multi-GPU split of the batched form, run as two gloo ranks on the CPU:
both ranks compute the same disjoint, complete, balanced split of the
64-system workload without communicating, and the step time is reduced
as the maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import workloads as W
from paper_2405_08737_gb300 import parallel


def _costs(seed=0):
    return [parallel.slice_cost(s["M"], s["n_t"] - 1) for s in W.batch_systems(64, seed)]


def test_shard_is_disjoint_complete_and_balanced():
    costs = _costs()
    for world in (1, 2, 3, 4, 8):
        shards = parallel.shard_systems(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in shards]
        ideal = max(sum(costs) / world, max(costs))
        assert max(loads) <= 4.0 / 3.0 * ideal, (world, max(loads) / ideal)


def test_shard_edge_cases():
    assert parallel.shard_systems([], 2) == [[], []]
    assert parallel.shard_systems([5.0], 3) == [[0], [], []]
    assert parallel.shard_systems([1.0, 1.0, 1.0, 1.0], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        parallel.shard_systems([1.0], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shards = parallel.shard_systems(_costs(), world)
        got = [None] * world
        dist.all_gather_object(got, shards[rank])
        t = parallel.max_over_ranks(10.0 + rank)
        out.put((rank, shards, got, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_split():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, shards, got, t in res:
        assert got == shards                 # every rank holds the same split
        assert t == 10.0 + world - 1         # max over ranks
    a, b = res[0][2]
    assert not set(a) & set(b) and sorted(a + b) == list(range(64))
