"""GPU parity of the thermal branch (Sec. 2, Eq. KBE3 and the tau terms of
Eq. KBE2) against the oracle's thermal runs: the rows of G^<, G^R and the
mixed rows G^|(t, tau) within 1e-12."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def kbe():
    import torch
    from paper_2405_08737_gb300 import build as B
    B.build()
    import paper_2405_08737_gb300 as K
    torch.cuda.set_device(0)
    return K


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = {  # name: (M, kind, U, pulse, beta, n_tau, k_tau, n_t, uniform)
    "free_dimer": (2, "goe", 0.0, False, 5.0, 41, 5, 21, True),
    "dimer_pulse": (2, "chain", 1.2, True, 4.0, 41, 5, 24, False),
    "goe4": (4, "goe", 0.8, False, 3.0, 33, 3, 18, False),
}


def _setup(name):
    M, kind, U, pulse_on, beta, N, kt, n_t, uniform = CASES[name]
    h = W.chain_h(M) if kind == "chain" else W.goe_h(M, 1)
    t, order = W.uniform_grid(n_t, 0.05, 5) if uniform else W.grid(n_t, 0.05, 0.3, 2)
    Uv = np.full(M, U)
    v = W.site_potential(M)
    pulse = dict(W.PULSE_CHAIN, t0=float(t[n_t // 2]), sigma=0.3) if pulse_on else None
    GM, rho, _ = W.thermal_free(h, beta, N)
    return M, h, t, order, Uv, v, pulse, beta, N, kt, GM, rho


def _gpu(kbe, name, precision="fp64"):
    M, h, t, order, Uv, v, pulse, beta, N, kt, GM, rho = _setup(name)
    n_t = len(t)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, Uv, v, pulse)
    ctx.set_thermal(beta, GM, k_tau=kt)
    run = kbe.Run(ctx)
    run.init_uncorrelated(rho)
    for n in range(1, n_t):
        run.step(n, P=2, precision=precision)
    ctx.sync_status()
    return ctx, run


@pytest.mark.parametrize("name", sorted(CASES))
def test_thermal_run_matches_oracle(kbe, name):
    M, h, t, order, Uv, v, pulse, beta, N, kt, GM, rho = _setup(name)
    Lo, Ro, Go = oracle.run_thermal(t, order, h, Uv, v, pulse, 2, beta, N, kt, GM, 1j * rho, -1j * np.eye(M),
                                    nthreads=4)
    ctx, run = _gpu(kbe, name)
    n_t = len(t)
    p = W.tri_size(n_t)
    assert _rel(run.L[:p].cpu().numpy(), Lo) < TOL
    assert _rel(run.R[:p].cpu().numpy(), Ro) < TOL
    assert _rel(ctx.mixed_rows(n_t).cpu().numpy(), Go) < TOL
    if name == "free_dimer":  # U = 0: the exact mixed function, to the stepper's accuracy
        _, _, mix = W.thermal_free(h, beta, N, t)
        assert np.abs(ctx.mixed_rows(n_t).cpu().numpy() - mix).max() < 2e-5
    ctx.close()


def test_thermal_split_precision(kbe):
    M, h, t, order, Uv, v, pulse, beta, N, kt, GM, rho = _setup("dimer_pulse")
    Lo, _, Go = oracle.run_thermal(t, order, h, Uv, v, pulse, 2, beta, N, kt, GM, 1j * rho, -1j * np.eye(M),
                                   nthreads=4)
    ctx, run = _gpu(kbe, "dimer_pulse", precision="split")
    assert _rel(run.L[:W.tri_size(len(t))].cpu().numpy(), Lo) < 5e-8
    assert _rel(ctx.mixed_rows(len(t)).cpu().numpy(), Go) < 5e-8
    ctx.close()


@pytest.mark.parametrize("name", ["dimer_pulse", "goe4"])
def test_thermal_double_float(kbe, name):
    """KBE_DF64 steps: the history slice and the two long thermal sums
    (mixed term, KBE3 history term) in double-float (about 2^-47 of the terms'
    sizes); the runs' rows stay within 1e-11 of the oracle's."""
    M, h, t, order, Uv, v, pulse, beta, N, kt, GM, rho = _setup(name)
    Lo, Ro, Go = oracle.run_thermal(t, order, h, Uv, v, pulse, 2, beta, N, kt, GM, 1j * rho, -1j * np.eye(M),
                                    nthreads=4)
    ctx, run = _gpu(kbe, name, precision="df64")
    p = W.tri_size(len(t))
    assert _rel(run.L[:p].cpu().numpy(), Lo) < 1e-11
    assert _rel(run.R[:p].cpu().numpy(), Ro) < 1e-11
    assert _rel(ctx.mixed_rows(len(t)).cpu().numpy(), Go) < 1e-11
    ctx.close()


def test_thermal_errors(kbe):
    import torch
    M, h, t, order, Uv, v, pulse, beta, N, kt, GM, rho = _setup("goe4")
    ctx = kbe.Context(M, len(t))
    ctx.set_grid(t, order)
    ctx.set_model(h, Uv, v, pulse)
    with pytest.raises(kbe.KBEError) as e:
        ctx.mixed_rows(2)
    assert e.value.status == kbe.KBE_ESTATE
    with pytest.raises(kbe.KBEError) as e:
        ctx.set_thermal(-1.0, GM)
    assert e.value.status == kbe.KBE_EINVAL
    ctx.set_thermal(beta, GM, k_tau=kt)
    with pytest.raises(kbe.KBEError) as e:
        ctx.set_interaction(W.coulomb_tensor(M, 1))
    assert e.value.status == kbe.KBE_EINVAL
    run = kbe.Run(ctx)
    run.init_uncorrelated(rho)
    run.step(1)
    with pytest.raises(kbe.KBEError) as e:
        kbe.Batch([run])
    assert e.value.status == kbe.KBE_EINVAL
    with pytest.raises(kbe.KBEError) as e:
        ctx.run_controlled(rho, 1e-6, 1e-8, 0.01, 1.0)
    assert e.value.status == kbe.KBE_ESTATE
    rows = ctx.mixed_rows(2)
    ctx.set_mixed_rows(rows)
    assert torch.equal(ctx.mixed_rows(2), rows)
    ctx.set_thermal(beta, None)
    ctx.sync_status()
    ctx.close()
