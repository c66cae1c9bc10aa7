"""GPU checks of adaptive history orders (Sec. 3.2): runs from the
uncorrelated state with the order of every interval chosen on the device,
against the oracle's adaptive runs (same chosen orders, rows to 1e-12)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

CASES = [  # (M, n_t, kind, seed, K, pulse)
    (2, 64, "chain", 0, 6, True), (3, 60, "goe", 1, 6, False), (8, 40, "chain", 2, 5, True),
    (4, 48, "goe", 3, 8, False),
]


@pytest.fixture(scope="module")
def kbe():
    import torch
    from paper_2405_08737_gb300 import build as B
    B.build()
    import paper_2405_08737_gb300 as K
    torch.cuda.set_device(0)
    return K


def _setup(M, n_t, kind, seed, with_pulse):
    t, order = W.grid(n_t, 0.05, 0.3, seed)
    h = W.chain_h(M, 1.0) if kind == "chain" else W.goe_h(M, seed)
    U = np.linspace(0.8, 1.6, M)
    v = W.site_potential(M)
    pulse = dict(W.PULSE_CHAIN, t0=float(t[n_t // 2]), sigma=0.4) if with_pulse else None
    return t, order, h, U, v, pulse


def _oracle_adaptive(t, order, h, U, v, pulse, K, P=2):
    M = h.shape[0]
    n_t = len(t)
    L0, R0, F0 = oracle.initial_rhs(t, order, h, U, v, pulse, W.half_filled_rho(h))
    L = np.zeros((W.tri_size(n_t), M, M), np.complex128)
    R = np.zeros_like(L)
    L[0], R[0] = L0[0], R0[0]
    Lo, Ro, _, hord = oracle.run_adaptive(t, order, [0], K, h, U, v, pulse, P, L, R, {0: F0}, 1, n_t, nthreads=4)
    return Lo, Ro, hord


def _gpu_adaptive(kbe, t, order, h, U, v, pulse, K, precision="fp64", P=2):
    M = h.shape[0]
    n_t = len(t)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, v, pulse)
    ctx.set_adaptive_orders(K)
    run = kbe.Run(ctx)
    run.init_uncorrelated(W.half_filled_rho(h))
    for n in range(1, n_t):
        run.step(n, P=P, precision=precision)
    ctx.sync_status()
    return ctx, run


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("case", CASES)
def test_adaptive_run_matches_oracle(kbe, case):
    M, n_t, kind, seed, K, with_pulse = case
    t, order, h, U, v, pulse = _setup(M, n_t, kind, seed, with_pulse)
    Lo, Ro, hord = _oracle_adaptive(t, order, h, U, v, pulse, K)
    ctx, run = _gpu_adaptive(kbe, t, order, h, U, v, pulse, K)
    ko = ctx.history_orders(n_t)
    assert np.array_equal(ko[1:], hord[1:n_t]), (ko, hord[:n_t])
    assert len(set(ko[K + 1:])) > 1  # the choice follows the data
    p = W.tri_size(n_t)
    assert _rel(run.L[:p].cpu().numpy(), Lo) < 1e-12
    assert _rel(run.R[:p].cpu().numpy(), Ro) < 1e-12
    ctx.close()


def test_adaptive_split_precision(kbe):
    M, n_t, kind, seed, K, with_pulse = CASES[2]
    t, order, h, U, v, pulse = _setup(M, n_t, kind, seed, with_pulse)
    Lo, _, _ = _oracle_adaptive(t, order, h, U, v, pulse, K)
    ctx, run = _gpu_adaptive(kbe, t, order, h, U, v, pulse, K, precision="split")
    assert _rel(run.L[:W.tri_size(n_t)].cpu().numpy(), Lo) < 5e-8  # compounded over the run
    ctx.close()


def test_adaptive_mode_errors_and_reset(kbe):
    M, n_t, kind, seed, K, with_pulse = CASES[1]
    t, order, h, U, v, pulse = _setup(M, n_t, kind, seed, with_pulse)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, v, pulse)
    with pytest.raises(kbe.KBEError) as e:
        ctx.set_adaptive_orders(13)
    assert e.value.status == kbe.KBE_ERANGE
    ctx.set_adaptive_orders(4)
    run = kbe.Run(ctx)
    run.init_uncorrelated(W.half_filled_rho(h))
    run.step(1)
    with pytest.raises(kbe.KBEError) as e:
        run.step(3)  # row 2 not stepped yet
    assert e.value.status == kbe.KBE_ESTATE
    run.step(2)
    run.step(2)  # stepping a row again is allowed
    with pytest.raises(kbe.KBEError) as e:
        kbe.Batch([run])
    assert e.value.status == kbe.KBE_EINVAL
    ctx.set_adaptive_orders(0)  # back to the grid's orders
    ko = ctx.history_orders(n_t)
    assert list(ko[1:]) == [min(int(order[l]), l) for l in range(1, n_t)]
    ctx.sync_status()
    ctx.close()
