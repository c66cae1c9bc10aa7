"""The batched form at the orbital counts and history lengths of the
64-system workload (M in {12, 16, 24}, rows of 150-260 points): one batched
KBE step of every system from a stored history, against the oracle's step
of each system, element by element.

The history rows 0..n-1 are the non-interacting propagators of each
system; both sides rebuild the stored right-hand-side rows n-K..n-1 from
them with their own code (kbe_rhs_row on the device, oracle.rhs_row on the
host), then take the step of row n (P = 2).  These lengths give history
chunks of several items for both tile sizes of the persistent FP64
kernel (128 and 256 output entries) and several 8-orbital parts in the
split contraction."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

SYSTEMS = [  # (M, n_t, kind, seed)
    (12, 200, "chain", 21), (16, 180, "goe", 22), (24, 160, "chain", 23), (4, 260, "goe", 24),
]


@pytest.fixture(scope="module")
def kbe():
    import torch
    from paper_2405_08737_gb300 import build as B
    B.build()
    import paper_2405_08737_gb300 as K
    torch.cuda.set_device(0)
    return K


def _model(M, n_t, kind, seed):
    t, order = W.grid(n_t, 0.02, 0.4, seed)
    h = W.chain_h(M, 1.0) if kind == "chain" else W.goe_h(M, seed)
    rng = np.random.default_rng(seed)
    U = rng.uniform(0.5, 3.0, M)
    return t, order, h, U, W.site_potential(M), None


@pytest.fixture(scope="module")
def oracle_rows():
    """Per system: the oracle's row n = n_t - 1 after its KBE step (P = 2)."""
    threads = oracle.threads_available()
    out = []
    for (M, n_t, kind, seed) in SYSTEMS:
        t, order, h, U, v, pulse = _model(M, n_t, kind, seed)
        n = n_t - 1
        Lh, Rh = W.free_triangles(h, W.half_filled_rho(h), t, n_rows=n)
        L = np.zeros((W.tri_size(n + 1), M, M), np.complex128)
        R = np.zeros_like(L)
        L[: W.tri_size(n)], R[: W.tri_size(n)] = Lh, Rh
        F = {j: oracle.rhs_row(j, t, order, h, U, v, pulse, L[: W.tri_size(j + 1)], R[: W.tri_size(j + 1)],
                               nthreads=threads)
             for j in oracle.f_rows_needed(order, n, n + 1)}
        Lo, Ro, _ = oracle.run(t, order, h, U, v, pulse, 2, L, R, F, n, n + 1, nthreads=threads)
        p = W.tri_size(n)
        out.append((Lo[p:p + n + 1], Ro[p:p + n + 1]))
    return out


def _runs(kbe):
    import torch
    runs = []
    for (M, n_t, kind, seed) in SYSTEMS:
        t, order, h, U, v, pulse = _model(M, n_t, kind, seed)
        ctx = kbe.Context(M, n_t)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, pulse)
        run = kbe.Run(ctx)
        n = n_t - 1
        Lh, Rh = W.free_triangles(h, W.half_filled_rho(h), t, n_rows=n)
        run.L[: W.tri_size(n)] = torch.as_tensor(Lh, device="cuda")
        run.R[: W.tri_size(n)] = torch.as_tensor(Rh, device="cuda")
        K = int(order[1:].max())
        for j in range(max(0, n - K), n):
            ctx.rhs_row(j, run.L, run.R, run.Sl, run.Sg, run.I, run.F)
        ctx.sync_status()
        runs.append(run)
    return runs


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _check_rows(runs, oracle_rows, tol):
    for run, (M, n_t, kind, seed), (Lo, Ro) in zip(runs, SYSTEMS, oracle_rows):
        n = n_t - 1
        p = W.tri_size(n)
        Lg = run.L[p:p + n + 1].cpu().numpy()
        Rg = run.R[p:p + n + 1].cpu().numpy()
        assert _rel(Lg, Lo) < tol, ((M, n_t), _rel(Lg, Lo))
        assert _rel(Rg, Ro) < tol, ((M, n_t), _rel(Rg, Ro))


@pytest.mark.parametrize("policy", ["autotuned", (128, 14), (256, 20)])
def test_batched_fp64_step_matches_oracle(kbe, oracle_rows, policy):
    runs = _runs(kbe)
    batch = kbe.Batch(runs)
    rows = [s[1] - 1 for s in SYSTEMS]
    if policy == "autotuned":
        blk, work, _ = batch.autotune(rows, reps=1)
        assert batch.policy() == (blk, work)
    else:
        batch.set_policy(*policy)
    batch.step(rows, P=2, precision="fp64")
    batch.sync_status()
    _check_rows(runs, oracle_rows, 1e-12)
    batch.close()
    for r in runs:
        r.ctx.close()


@pytest.mark.parametrize("precision,tol", [("split", 1e-8), ("df64", 1e-11)])
def test_batched_step_other_precisions_match_oracle(kbe, oracle_rows, precision, tol):
    runs = _runs(kbe)
    batch = kbe.Batch(runs)
    batch.step([s[1] - 1 for s in SYSTEMS], P=2, precision=precision)
    batch.sync_status()
    _check_rows(runs, oracle_rows, tol)
    batch.close()
    for r in runs:
        r.ctx.close()
