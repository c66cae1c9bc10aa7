"""GPU checks of the batched form: independent systems of different orbital
counts and grid lengths advanced by one graph launch per step, against the
oracle's run of each system and against the single-system stepper."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

SYSTEMS = [  # (M, n_t, kind, seed)
    (1, 20, "chain", 1), (2, 33, "chain", 2), (3, 41, "goe", 3), (4, 28, "chain", 4),
    (5, 37, "goe", 5), (8, 24, "chain", 6),
]


@pytest.fixture(scope="module")
def kbe():
    import torch
    from paper_2405_08737_gb300 import build as B
    B.build()
    import paper_2405_08737_gb300 as K
    torch.cuda.set_device(0)
    return K


def _system(M, n_t, kind, seed):
    t, order = W.grid(n_t, 0.05, 0.4, seed)
    h = W.chain_h(M, 1.0) if kind == "chain" else W.goe_h(M, seed)
    rng = np.random.default_rng(seed)
    U = rng.uniform(0.5, 3.0, M)
    v = W.site_potential(M)
    pulse = dict(W.PULSE_CHAIN, t0=float(t[n_t // 2]), sigma=0.3) if seed % 2 == 0 else None
    return t, order, h, U, v, pulse


def _runs(kbe, systems=SYSTEMS):
    out = []
    for (M, n_t, kind, seed) in systems:
        t, order, h, U, v, pulse = _system(M, n_t, kind, seed)
        ctx = kbe.Context(M, n_t)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, pulse)
        run = kbe.Run(ctx)
        run.init_uncorrelated(W.half_filled_rho(h))
        out.append(run)
    return out


def _oracle(M, n_t, kind, seed, P=2):
    t, order, h, U, v, pulse = _system(M, n_t, kind, seed)
    L0, R0, F0 = oracle.initial_rhs(t, order, h, U, v, pulse, W.half_filled_rho(h))
    Lo = np.zeros((W.tri_size(n_t), M, M), np.complex128)
    Ro = np.zeros_like(Lo)
    Lo[0], Ro[0] = L0[0], R0[0]
    Lo, Ro, _ = oracle.run(t, order, h, U, v, pulse, P, Lo, Ro, {0: F0}, 1, n_t, nthreads=4)
    return Lo, Ro


def _advance(batch, systems, precision="fp64", P=2, upto=None):
    n_end = max(s[1] for s in systems) if upto is None else upto
    for n in range(1, n_end):
        rows = [n if n < s[1] else -1 for s in systems]
        batch.step(rows, P=P, precision=precision)
    batch.sync_status()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("policy", [(256, 20), (128, 14), (256, 26)])
def test_batch_matches_oracle(kbe, policy):
    runs = _runs(kbe)
    batch = kbe.Batch(runs)
    batch.set_policy(*policy)
    _advance(batch, SYSTEMS)
    for run, s in zip(runs, SYSTEMS):
        Lo, Ro = _oracle(*s)
        n_t = s[1]
        Lg = run.L[: W.tri_size(n_t)].cpu().numpy()
        Rg = run.R[: W.tri_size(n_t)].cpu().numpy()
        assert _rel(Lg, Lo) < 1e-12, (s, _rel(Lg, Lo))
        assert _rel(Rg, Ro) < 1e-12, (s, _rel(Rg, Ro))
    batch.close()


def test_batch_matches_single_system_stepper(kbe):
    runs = _runs(kbe)
    batch = kbe.Batch(runs)
    _advance(batch, SYSTEMS)
    single = _runs(kbe)
    for run, s in zip(single, SYSTEMS):
        for n in range(1, s[1]):
            run.step(n, P=2)
        run.ctx.sync_status()
    for a, b, s in zip(runs, single, SYSTEMS):
        p = W.tri_size(s[1])
        err = _rel(a.L[:p].cpu().numpy(), b.L[:p].cpu().numpy())
        assert err < 1e-13, (s, err)
    batch.close()


def test_batch_split_precision(kbe):
    """The split-precision bound is per slice: one batched split step from
    an FP64 history matches the oracle's step to 1e-8 in every system.  A
    whole run with the split contraction compounds one slice error per step
    (about 40 steps here); it is checked at 5e-8."""
    runs = _runs(kbe)
    batch = kbe.Batch(runs)
    n_last = max(s[1] for s in SYSTEMS) - 1
    for n in range(1, n_last):
        batch.step([n if n < s[1] - 1 else -1 for s in SYSTEMS], P=2, precision="fp64")
    batch.step([s[1] - 1 for s in SYSTEMS], P=2, precision="split")
    batch.sync_status()
    for run, s in zip(runs, SYSTEMS):
        Lo, _ = _oracle(*s)
        n = s[1] - 1
        p = W.tri_size(n)
        Lg = run.L[p:p + n + 1].cpu().numpy()
        assert _rel(Lg, Lo[p:p + n + 1]) < 1e-8, (s, _rel(Lg, Lo[p:p + n + 1]))
    batch.close()
    runs = _runs(kbe)
    batch = kbe.Batch(runs)
    _advance(batch, SYSTEMS, precision="split")
    for run, s in zip(runs, SYSTEMS):
        Lo, _ = _oracle(*s)
        Lg = run.L[: W.tri_size(s[1])].cpu().numpy()
        assert _rel(Lg, Lo) < 5e-8, (s, _rel(Lg, Lo))
    batch.close()


def test_batch_double_float(kbe):
    """Batched KBE_DF64 steps run each system's double-float slice in the
    graph: whole runs match the single-system KBE_DF64 stepper (1e-13) and
    the oracle (1e-11)."""
    runs = _runs(kbe)
    batch = kbe.Batch(runs)
    _advance(batch, SYSTEMS, precision="df64")
    single = _runs(kbe)
    for run, s in zip(single, SYSTEMS):
        for n in range(1, s[1]):
            run.step(n, P=2, precision="df64")
        run.ctx.sync_status()
    for a, b, s in zip(runs, single, SYSTEMS):
        p = W.tri_size(s[1])
        La = a.L[:p].cpu().numpy()
        assert _rel(La, b.L[:p].cpu().numpy()) < 1e-13, s
        Lo, _ = _oracle(*s)
        assert _rel(La, Lo) < 1e-11, (s, _rel(La, Lo))
    batch.close()


def test_batch_inactive_systems_untouched_and_graph_reused(kbe):
    import torch
    runs = _runs(kbe)
    batch = kbe.Batch(runs)
    systems = SYSTEMS
    for n in range(1, 6):
        batch.step([n] * len(systems))
    counts = set()
    frozen = runs[2].L.clone(), runs[2].F.clone()
    for n in range(6, 12):
        rows = [n] * len(systems)
        rows[2] = -1
        batch.step(rows)
        counts.add(batch.last_launch_count)
    batch.sync_status()
    assert torch.equal(runs[2].L, frozen[0]) and torch.equal(runs[2].F, frozen[1])
    # one graph of plan + predictor + P x 7 kernels, reused for every step
    assert counts == {2 + 2 * 7}
    batch.close()


def test_batch_autotune_and_errors(kbe):
    runs = _runs(kbe)
    batch = kbe.Batch(runs)
    _advance(batch, SYSTEMS, upto=12)
    rows = [s[1] - 1 for s in SYSTEMS]
    block, work, ms = batch.autotune([11] * len(SYSTEMS), reps=1)
    assert block in (128, 256) and 14 <= work <= 26 and ms > 0
    assert batch.policy() == (block, work)
    with pytest.raises(kbe.KBEError) as e:
        batch.step([s[1] for s in SYSTEMS])
    assert e.value.status == kbe.KBE_ERANGE
    with pytest.raises(kbe.KBEError) as e:
        batch.set_policy(64, 20)
    assert e.value.status == kbe.KBE_EINVAL
    del rows
    batch.close()


def test_batch_precisions_alternate_on_the_same_rows(kbe):
    """A split step right after an FP64 step of the same rows (and the FP64
    step again after it) rebuilds the split work list for those rows: each
    step matches the single-system stepper in its precision."""
    runs = _runs(kbe)
    batch = kbe.Batch(runs)
    _advance(batch, SYSTEMS, upto=10)
    rows = [min(10, s[1] - 1) for s in SYSTEMS]
    single = _runs(kbe)
    for run, s in zip(single, SYSTEMS):
        for n in range(1, 10):
            run.step(n, P=2)
    for prec, tol in (("fp64", 1e-13), ("split", 1e-12), ("fp64", 1e-13)):
        batch.step(rows, P=2, precision=prec)
        batch.sync_status()
        for a, b, n in zip(runs, single, rows):
            b.ctx.set_split_planes(False)
            b.step(n, P=2, precision=prec)
            b.ctx.sync_status()
            p = W.tri_size(n)
            err = _rel(a.L[p:p + n + 1].cpu().numpy(), b.L[p:p + n + 1].cpu().numpy())
            assert err < tol, (prec, n, err)
    batch.close()
