"""Host-side work split for one process per GPU.

The systems of a batched step are independent, so N GPUs share a batch by
taking disjoint sets of systems: no collective touches the data path, and
only the step time is reduced (the maximum over ranks).

One system can be split too: the stored triangle is cut into contiguous
bands of rows, one per rank, with about equal numbers of stored blocks
(row_bands); each rank's device computes its band's contributions with
Context.history_slice_band (kbe_history_slice_band), and sharded_slice sums
them; sharded_step runs a whole KBE step of such a system (the predictor,
then per sweep the self-energy row and the band's partial slice, the
all-reduce, and the Fock matrix, right-hand side and corrector, which every
rank forms identically from the reduced slice).  The host logic is tested with gloo ranks on the CPU and the per-band
kernel on one GPU (the bands one after another); no call here drives more
than one GPU.  A stored block (r, c), r >= c, enters the history
slice of row n (Eq. KBE2) three times: term 1 of output column c (history
point m = r), term 1 of output column r through G(c, r) = -G(r, c)^+ (m = c,
r != c) and term 2 of output column r through G^A(c, r) = R(r, c)^+ (m = c).
So each rank adds the contributions of its own blocks to all n + 1 output
columns, and one all-reduce of the 2 (n+1) M^2 complex partials gives every
rank the slice; the self-energy row n and the new row n itself are O(n M^2)
and every rank computes them from the reduced slice.  Communication is
O(n M^2) per slice against O(n^2 M^3 / N) work per rank.  The split balances
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


def tri(n):
    """Stored blocks of rows 0..n-1 of a lower triangle: n (n+1) / 2."""
    return n * (n + 1) // 2


def row_bands(n_rows, world):
    """Contiguous bands [lo, hi) of the rows 0..n_rows-1, one per rank, each
    holding about tri(n_rows) / world stored blocks (row r holds r + 1
    blocks); deterministic, so every rank derives the same bands."""
    if world < 1:
        raise ValueError("world must be >= 1")
    total = tri(n_rows)
    bounds = [0]
    for k in range(1, world):
        target = total * k / world
        r = bounds[-1]
        while r < n_rows and tri(r + 1) <= target:
            r += 1
        # the nearer of r and r + 1 to the target, never before the last bound
        if r < n_rows and abs(tri(r + 1) - target) < abs(tri(r) - target):
            r += 1
        bounds.append(max(bounds[-1], r))
    bounds.append(n_rows)
    return [(bounds[k], bounds[k + 1]) for k in range(world)]


def band_owner(bands, r):
    """The rank whose band holds row r."""
    for k, (lo, hi) in enumerate(bands):
        if lo <= r < hi:
            return k
    raise ValueError("row %d is in no band" % r)


def sharded_slice(partial, group=None):
    """Sum the ranks' partial history slices in place (all-reduce over
    ``group``); every rank ends with the whole slice.  ``partial`` holds this
    rank's contributions [2][n+1][M][M] (complex128, on the rank's device)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(partial, op=dist.ReduceOp.SUM, group=group)
    return partial



def sharded_step(ctx, n, P, band, L, R, Sl, Sg, I, F, group=None, stream=None):
    """One KBE step (KBE_FP64) of row n of a system whose stored rows are
    split in bands across ranks: ``band`` = (lo, hi) is this rank's rows
    (row_bands), L, R, Sl, Sg, I, F the buffers of kbe_step on this rank's
    device.  The predictor, then P sweeps of {self-energy row n and the
    band's partial slice (kbe_step_sweep_band), all-reduce of the
    2 (n+1) M^2 partials (sharded_slice), Fock matrix, right-hand side and
    corrector (kbe_step_sweep_finish)}.  Every rank forms row n from the same
    reduced slice, so no row is broadcast; a rank reads only its band's rows
    of the history, rows n-1 and n, and the right-hand-side ring.  With one
    rank and the band (0, n+1) this is kbe_step, bitwise.  Returns the
    numbers of all-reduces (P) and of the kernels the phases launched."""
    import torch
    lo, hi = min(int(band[0]), n + 1), min(int(band[1]), n + 1)
    M = ctx.M
    size = 2 * (n + 1) * M * M
    flat = I.reshape(-1)[:size]
    kernels = 0
    ctx.step_predict(n, L, R, F, stream=stream)
    kernels += getattr(ctx, "last_launch_count", 0)
    for _ in range(P):
        ctx.step_sweep_band(n, lo, hi, L, R, Sl, Sg, I, stream=stream)
        kernels += getattr(ctx, "last_launch_count", 0)
        sharded_slice(torch.view_as_real(flat) if flat.is_complex() else flat, group)
        ctx.step_sweep_finish(n, L, R, I, F, stream=stream)
        kernels += getattr(ctx, "last_launch_count", 0)
    return {"all_reduces": P, "kernels": kernels}
