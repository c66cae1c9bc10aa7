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


# ------------------------------------------------ one system, whole step --
# parallel.sharded_step drives the phases of a KBE step (kbe_step_predict,
# kbe_step_sweep_band, kbe_step_sweep_finish) and the all-reduce.  On the CPU
# the phases are played by _HostPhases, written here from the stepper's
# formulas (include/kbe.h, kbe_step): the band's partial slice of Eq. (KBE2)
# as above, the predictor and corrector of the integral-form Adams rules,
# and F^s(n,c) = -i(eps(t_n) G^s(n,c) + I^s(n,c)) with the oracle's Fock
# matrix.  The ranks' whole step must equal the oracle's step to 1e-12.

class _HostPhases:
    def __init__(self, t, order, h, U, v, pulse, F):
        import oracle
        self.oracle = oracle
        self.t, self.order, self.h, self.U, self.v, self.pulse = t, order, h, U, v, pulse
        self.M = h.shape[0]
        self.F = dict(F)  # row j -> [2, j+1, M, M]
        self.calls = []

    def _w(self, first, last, n):
        return self.oracle.lagrange_weights(self.t[first:last + 1], self.t[n - 1], self.t[n])

    def _step_rows(self, n, L, R, rows):
        """G(n, .) = G(n-1, .) + sum_p w_p F(row_p, .) over the rows of the rule."""
        M, kn = self.M, int(self.order[n])
        tri = W.tri_index
        Gl = np.zeros((n + 1, M, M), np.complex128)
        Gg = np.zeros_like(Gl)
        for c in range(n):
            q = min(kn, n - c)
            first, last = rows(q)
            w = self._w(first, last, n)
            al = L[tri(n - 1, c)].copy()
            ag = R[tri(n - 1, c)] + L[tri(n - 1, c)]
            for p, j in enumerate(range(first, last + 1)):
                al = al + w[p] * self.F[j][0, c]
                ag = ag + w[p] * self.F[j][1, c]
            Gl[c], Gg[c] = al, ag
        q = min(kn, n)
        first, last = rows(q)
        w = self._w(first, last, n)
        al = L[tri(n - 1, n - 1)].copy()
        for p, j in enumerate(range(first, last + 1)):
            D = self.F[j][0, j] - self.F[j][0, j].conj().T  # d G^<(t,t)/dt at t_j
            al = al + w[p] * D
        Gl[n] = al
        for c in range(n):
            L[tri(n, c)] = Gl[c]
            R[tri(n, c)] = Gg[c] - Gl[c]
        L[tri(n, n)] = Gl[n]
        R[tri(n, n)] = -1j * np.eye(M)

    def step_predict(self, n, L, R, F, stream=None):
        self.calls.append(("predict", n))
        self._step_rows(n, L, R, lambda q: (n - q, n - 1))

    def step_sweep_band(self, n, lo, hi, L, R, Sl, Sg, I, stream=None):
        import torch
        self.calls.append(("band", n, lo, hi))
        sl, sg = self.oracle.sigma_row(self.oracle.local_U4(self.U), n, L, R)
        Sl[: n + 1], Sg[: n + 1] = sl, sg
        part = _band_contributions(self.t, self.order, n, L, R, sl, sg, (lo, hi))
        I.reshape(-1)[: part.size] = torch.from_numpy(part.ravel())

    def step_sweep_finish(self, n, L, R, I, F, stream=None):
        self.calls.append(("finish", n))
        M = self.M
        Iv = I.reshape(-1)[: 2 * (n + 1) * M * M].numpy().reshape(2, n + 1, M, M)
        eps = self.oracle.fock(self.t[n], self.h, self.U, self.v, self.pulse, L[W.tri_index(n, n)])
        Fn = np.zeros((2, n + 1, M, M), np.complex128)
        for c in range(n + 1):
            Gl = L[W.tri_index(n, c)]
            Gg = R[W.tri_index(n, c)] + Gl
            Fn[0, c] = -1j * (eps @ Gl + Iv[0, c])
            Fn[1, c] = -1j * (eps @ Gg + Iv[1, c])
        self.F[n] = Fn
        self._step_rows(n, L, R, lambda kap: (n - kap, n))


def _step_case():
    import oracle
    M, n_t, seed = 3, 13, 9
    t, order = W.grid(n_t, 0.05, 0.4, seed)
    h = W.goe_h(M, seed)
    U, v = np.linspace(0.5, 1.5, M), W.site_potential(M)
    pulse = {"E0": 0.4, "t0": float(t[n_t // 2]), "sigma": 0.3, "omega": 2.0}
    n = n_t - 1
    Lh, Rh, F = W.restart_state(h, W.half_filled_rho(h), t, order, n, n)
    L = np.zeros((W.tri_size(n + 1), M, M), np.complex128)
    R = np.zeros_like(L)
    L[: W.tri_size(n)], R[: W.tri_size(n)] = Lh, Rh
    Lo, Ro, Io = oracle.run(t, order, h, U, v, pulse, 2, L, R, F, n, n + 1)
    return (t, order, h, U, v, pulse, n, L, R, F), (Lo, Ro)


def _step_rank(rank, world, port, case, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, order, h, U, v, pulse, n, L, R, F = case
        L, R = L.copy(), R.copy()
        M = h.shape[0]
        ph = _HostPhases(t, order, h, U, v, pulse, F)
        bands = parallel.row_bands(n + 1, world)
        Sl = np.zeros((n + 1, M, M), np.complex128)
        Sg = np.zeros_like(Sl)
        I = torch.zeros((2, n + 1, M, M), dtype=torch.complex128)
        reduces = parallel.sharded_step(ph, n, 2, bands[rank], L, R, Sl, Sg, I, None)
        p = W.tri_size(n)
        out.put((rank, bands, ph.calls, reduces, L[p:p + n + 1], R[p:p + n + 1]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 3])
def test_sharded_step_ranks_match_the_oracle_step(world):
    """Every rank runs predictor, P = 2 sweeps of {band partial slice,
    all-reduce, finish} on its row band; each rank's new row n equals the
    oracle's KBE step of row n to 1e-12, and the ranks agree bitwise."""
    case, (Lo, Ro) = _step_case()
    n = case[6]
    p = W.tri_size(n)
    port = _free_port()
    mctx = mp.get_context("spawn")
    q = mctx.Queue()
    procs = [mctx.Process(target=_step_rank, args=(r, world, port, case, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted([q.get(timeout=180) for _ in range(world)], key=lambda x: x[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    scale = max(np.abs(Lo[p:]).max(), np.abs(Ro[p:]).max())
    for rank, bands, calls, reduces, Ln, Rn in res:
        lo, hi = bands[rank]
        assert calls == [("predict", n), ("band", n, lo, hi), ("finish", n), ("band", n, lo, hi), ("finish", n)]
        assert reduces["all_reduces"] == 2
        assert np.abs(Ln - Lo[p:]).max() <= 1e-12 * scale, (world, rank, np.abs(Ln - Lo[p:]).max() / scale)
        assert np.abs(Rn - Ro[p:]).max() <= 1e-12 * scale
        assert np.array_equal(Ln, res[0][4]) and np.array_equal(Rn, res[0][5])
