"""The multi-GPU splits, run as gloo ranks on the CPU.

Batched form: both ranks compute the same disjoint, complete, balanced split
of the 64-system workload without communicating, and the step time is
reduced as the maximum over ranks.  One system: the ranks' row-band
contributions, summed by one all-reduce, give the oracle's history slice."""
import os
import socket

import numpy as np
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


# ------------------------------------------------- one system, row bands --
# The plan for one system on several GPUs: rows in contiguous bands, each
# rank adds the contributions of its stored blocks to every output column,
# one all-reduce sums them.  The per-rank contributions below are written
# from Eq. (KBE2) for this test (the library's kernels run on one GPU); the
# sum over ranks must be the oracle's slice.

def _band_contributions(t, order, n, L, R, Sl, Sg, band):
    """Contributions of the stored blocks (r, c), r in band, r <= n, to the
    slice of row n: term 1 of column c (m = r), term 1 of column r through
    G(c, r) = -G(r, c)^+ (m = c < r), term 2 of column r through
    G^A(c, r) = R(r, c)^+ (m = c)."""
    import oracle
    M = L.shape[-1]
    out = np.zeros((2, n + 1, M, M), np.complex128)
    wn = oracle.composite_row(t, order, n)
    SR = Sg - Sl
    S = (Sl, Sg)
    lo, hi = band
    for r in range(lo, min(hi, n + 1)):
        wr = oracle.composite_row(t, order, r)
        for c in range(r + 1):
            Lb, Rb = L[W.tri_index(r, c)], R[W.tri_index(r, c)]
            G = (Lb, Lb + Rb)  # G^<(r, c), G^>(r, c)
            for s in range(2):
                out[s, c] += wn[r] * SR[r] @ G[s]
                if r != c:
                    out[s, r] += wn[c] * SR[c] @ (-G[s].conj().T)
                out[s, r] += wr[c] * S[s][c] @ Rb.conj().T
    return out


def _band_rank(rank, world, port, case, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, order, n, L, R, Sl, Sg = case
        bands = parallel.row_bands(n + 1, world)
        part = torch.from_numpy(_band_contributions(t, order, n, L, R, Sl, Sg, bands[rank]))
        parallel.sharded_slice(part)
        out.put((rank, bands, part.numpy()))
    finally:
        dist.destroy_process_group()


def test_row_bands_partition_and_balance():
    for n_rows in (1, 2, 7, 64, 1024):
        for world in (1, 2, 3, 4, 8):
            bands = parallel.row_bands(n_rows, world)
            assert len(bands) == world and bands[0][0] == 0 and bands[-1][1] == n_rows
            assert all(bands[k][1] == bands[k + 1][0] for k in range(world - 1))
            blocks = [parallel.tri(hi) - parallel.tri(lo) for lo, hi in bands]
            # within one row (at most n_rows blocks) of the even share
            assert max(blocks) - parallel.tri(n_rows) / world <= n_rows, (n_rows, world, blocks)
            assert all(parallel.band_owner(bands, r) in range(world) for r in range(n_rows))
    with pytest.raises(ValueError):
        parallel.row_bands(4, 0)


@pytest.mark.parametrize("world,kind", [(2, "free"), (3, "random")])
def test_row_band_ranks_sum_to_the_oracle_slice(world, kind):
    import oracle
    M, n_t, seed = 3, 14, 4
    t, order = W.grid(n_t, 0.05, 0.4, seed)
    if kind == "free":
        h = W.goe_h(M, seed)
        L, R = W.free_triangles(h, W.half_filled_rho(h), t)
    else:
        L, R = W.random_triangles(M, n_t, seed)
    n = n_t - 1
    Sl, Sg = oracle.sigma_row(oracle.local_U4(np.linspace(0.5, 1.5, M)), n, L, R)
    ref = oracle.history_slice(t, order, n, L, R, Sl, Sg)
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    case = (t, order, n, L, R, Sl, Sg)
    procs = [ctx.Process(target=_band_rank, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    scale = np.abs(ref).max()
    for rank, bands, got in res:
        assert bands == parallel.row_bands(n + 1, world)
        assert np.abs(got - ref).max() <= 1e-12 * scale, (rank, np.abs(got - ref).max() / scale)
