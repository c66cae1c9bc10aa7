"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerance: 1e-12 relative in the max norm per slice (both s, all columns)
for the FP64 path.  The self-energy kernel forms its products in
double-float arithmetic (about 2^-47 per operation, a few 1e-14 per entry)
and is checked at 1e-13."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
TOL_SIGMA = 1e-13


@pytest.fixture(scope="module")
def kbe():
    import torch
    from paper_2405_08737_gb300 import build as B
    B.build()
    import paper_2405_08737_gb300 as K
    torch.cuda.set_device(0)
    return K


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _case(M, n_t, seed, kind="free", kmax=5):
    t, order = W.grid(n_t, 0.05, 0.4, seed, kmax=kmax)
    h = W.goe_h(M, seed)
    rho0 = W.half_filled_rho(h)
    if kind == "free":
        L, R = W.free_triangles(h, rho0, t)
    else:
        L, R = W.random_triangles(M, n_t, seed)
    U = np.linspace(0.5, 1.5, M)
    return t, order, h, rho0, U, L, R


def _ctx(kbe, M, n_max, t, order, h, U):
    ctx = kbe.Context(M, n_max)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, W.site_potential(M), None)
    return ctx


@pytest.mark.parametrize("M,n_t,n", [(1, 4, 0), (2, 12, 5), (3, 20, 19), (8, 70, 63), (5, 33, 20)])
def test_sigma_slice(kbe, M, n_t, n):
    import torch
    t, order, h, rho0, U, L, R = _case(M, n_t, M + n)
    ctx = _ctx(kbe, M, n_t, t, order, h, U)
    Ld, Rd = _dev(L), _dev(R)
    Sl = torch.zeros((n + 1, M, M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    ctx.selfenergy_slice(n, Ld, Rd, Sl, Sg)
    ctx.sync_status()
    ol, og = oracle.sigma_row(oracle.local_U4(U), n, L, R)
    assert _rel(Sl.cpu().numpy(), ol) < TOL_SIGMA
    assert _rel(Sg.cpu().numpy(), og) < TOL_SIGMA
    assert ctx.last_launch_count == 0  # sync_status launches nothing


def test_sigma_all_rows(kbe):
    import torch
    M, n_t = 3, 20
    t, order, h, rho0, U, L, R = _case(M, n_t, 4)
    ctx = _ctx(kbe, M, n_t, t, order, h, U)
    Sl = torch.zeros((W.tri_size(n_t), M, M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    ctx.selfenergy_all(n_t, _dev(L), _dev(R), Sl, Sg)
    ctx.sync_status()
    Sl, Sg = Sl.cpu().numpy(), Sg.cpu().numpy()
    for n in range(n_t):
        ol, og = oracle.sigma_row(oracle.local_U4(U), n, L, R)
        p = W.tri_index(n, 0)
        assert _rel(Sl[p:p + n + 1], ol) < TOL_SIGMA
        assert _rel(Sg[p:p + n + 1], og) < TOL_SIGMA


def _gpu_slice(kbe, ctx, n, L, R, Sl, Sg):
    import torch
    M = ctx.M
    out = torch.zeros((2, n + 1, M, M), dtype=torch.complex128, device="cuda")
    ctx.history_slice(n, L, R, _dev(Sl) if isinstance(Sl, np.ndarray) else Sl,
                      _dev(Sg) if isinstance(Sg, np.ndarray) else Sg, out)
    ctx.sync_status()
    return out.cpu().numpy()


@pytest.mark.parametrize("M", [1, 2, 3, 5, 8, 16])
@pytest.mark.parametrize("kind", ["free", "random"])
def test_history_slice_small(kbe, M, kind):
    n_t = 40
    t, order, h, rho0, U, L, R = _case(M, n_t, 7 * M, kind)
    ctx = _ctx(kbe, M, n_t, t, order, h, U)
    Ld, Rd = _dev(L), _dev(R)
    for n in (0, 1, 2, 5, 17, 39):
        if kind == "free":
            Sl, Sg = oracle.sigma_row(oracle.local_U4(U), n, L, R)
        else:
            Sl, Sg = W.random_rows(M, n, 3 * n + M)
        I = _gpu_slice(kbe, ctx, n, Ld, Rd, Sl, Sg)
        ref = oracle.history_slice(t, order, n, L, R, Sl, Sg, nthreads=8)
        assert _rel(I, ref) < TOL, (M, kind, n, _rel(I, ref))


def test_history_slice_high_orders(kbe):
    M, n_t = 4, 60
    t, order, h, rho0, U, L, R = _case(M, n_t, 3, "free", kmax=12)
    ctx = _ctx(kbe, M, n_t, t, order, h, U)
    Ld, Rd = _dev(L), _dev(R)
    for n in (3, 12, 13, 59):
        Sl, Sg = oracle.sigma_row(oracle.local_U4(U), n, L, R)
        I = _gpu_slice(kbe, ctx, n, Ld, Rd, Sl, Sg)
        ref = oracle.history_slice(t, order, n, L, R, Sl, Sg, nthreads=8)
        assert _rel(I, ref) < 1e-11, n  # high-order weights differ by ~1e-13 between routes


def test_history_all_slices_dimer(kbe):
    """Hubbard dimer, 64 nonuniform points, orders in {1..5}: every slice."""
    cfg = W.CONFIGS["dimer_m2_n64"]
    t, order = W.grid(cfg["n_t"], cfg["dt0"], cfg["sig"], 0)
    h, U, v, pulse = W.build_model(cfg, 0)
    rho0 = W.half_filled_rho(h)
    L, R = W.free_triangles(h, rho0, t)
    M = cfg["M"]
    ctx = _ctx(kbe, M, cfg["n_t"], t, order, h, U)
    Ld, Rd = _dev(L), _dev(R)
    import torch
    Sl = torch.zeros((cfg["n_t"], M, M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    for n in range(cfg["n_t"]):
        ctx.selfenergy_slice(n, Ld, Rd, Sl, Sg)
        I = _gpu_slice(kbe, ctx, n, Ld, Rd, Sl[: n + 1].contiguous(), Sg[: n + 1].contiguous())
        ol, og = oracle.sigma_row(oracle.local_U4(U), n, L, R)
        ref = oracle.history_slice(t, order, n, L, R, ol, og, nthreads=8)
        assert _rel(I, ref) < TOL, n


def _full_size_case(kbe, name, seed=0):
    import torch
    cfg = W.CONFIGS[name]
    M, n_t = cfg["M"], cfg["n_t"]
    t, order = W.grid(n_t, cfg["dt0"], cfg["sig"], seed)
    h, U, v, pulse = W.build_model(cfg, seed)
    rho0 = W.half_filled_rho(h)
    Ld, Rd = W.free_triangles_torch(h, rho0, t, n_t, "cuda")
    ctx = _ctx(kbe, M, n_t, t, order, h, U)
    return cfg, t, order, h, U, ctx, Ld, Rd


@pytest.mark.parametrize("name", ["chain_m8_n1024"])
def test_history_full_size_sampled(kbe, name):
    """The full-size slice n = N_t - 1 in the launch configuration the
    benchmark times; the oracle evaluates sampled output columns."""
    import torch
    cfg, t, order, h, U, ctx, Ld, Rd = _full_size_case(kbe, name)
    M, n = cfg["M"], cfg["n_t"] - 1
    Sl = torch.zeros((n + 1, M, M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    ctx.selfenergy_slice(n, Ld, Rd, Sl, Sg)
    out = torch.zeros((2, n + 1, M, M), dtype=torch.complex128, device="cuda")
    ctx.history_slice(n, Ld, Rd, Sl, Sg, out)
    ctx.sync_status()
    I = out.cpu().numpy()
    L, R = Ld.cpu().numpy(), Rd.cpu().numpy()
    Sl_h, Sg_h = Sl.cpu().numpy(), Sg.cpu().numpy()
    ol, og = oracle.sigma_row(oracle.local_U4(U), n, L, R)
    assert _rel(Sl_h, ol) < TOL_SIGMA and _rel(Sg_h, og) < TOL_SIGMA
    cols = [0, 1, 2, 255, 511, 700, n - 5, n - 1, n]
    ref = oracle.history_columns(t, order, n, L, R, ol, og, cols, nthreads=oracle.threads_available())
    assert _rel(I[:, cols], ref) < TOL


def _oracle_run(t, order, h, U, v, pulse, rho0, n_t, P=2):
    M = h.shape[0]
    L0, R0, F0 = oracle.initial_rhs(t, order, h, U, v, pulse, rho0)
    L = np.zeros((W.tri_size(n_t), M, M), np.complex128)
    R = np.zeros_like(L)
    L[0], R[0] = L0[0], R0[0]
    return oracle.run(t[:n_t], order[:n_t], h, U, v, pulse, P, L, R, {0: F0}, 1, n_t,
                      nthreads=oracle.threads_available())


@pytest.mark.parametrize("name,n_t", [("dimer_m2_n64", 64), ("chain_m8_n1024", 48)])
def test_stepper_matches_oracle(kbe, name, n_t):
    cfg = W.CONFIGS[name]
    t, order = W.grid(cfg["n_t"], cfg["dt0"], cfg["sig"], 1)
    t, order = t[:n_t], order[:n_t]
    h, U, v, pulse = W.build_model(cfg, 1)
    if pulse is not None:  # move the pulse into the short window
        pulse = dict(pulse, t0=t[n_t // 2], sigma=0.3)
    rho0 = W.half_filled_rho(h)
    M = cfg["M"]
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, v, pulse)
    run = kbe.Run(ctx)
    run.init_uncorrelated(rho0)
    for n in range(1, n_t):
        run.step(n, P=2)
    ctx.sync_status()
    Lo, Ro, Io = _oracle_run(t, order, h, U, v, pulse, rho0, n_t)
    L, R = run.L.cpu().numpy(), run.R.cpu().numpy()
    for n in range(n_t):
        p = W.tri_index(n, 0)
        assert _rel(L[p:p + n + 1], Lo[p:p + n + 1]) < TOL, n
        assert _rel(R[p:p + n + 1], Ro[p:p + n + 1]) < TOL, n
    # last history slice as well
    assert _rel(run.I[:, :n_t].cpu().numpy(), Io) < TOL


def test_restart_from_frozen_history(kbe):
    """Restart at row ns from a non-interacting history with its exact
    right-hand sides (the frozen state of the gradient window)."""
    import torch
    cfg = W.CONFIGS["chain_m16_n512_w32"]
    M, n_t, ns = cfg["M"], 40, 32
    t, order = W.grid(cfg["n_t"], cfg["dt0"], cfg["sig"], 2)
    t, order = t[:n_t], order[:n_t]
    h, U, v, pulse = W.build_model(cfg, 2)
    pulse = dict(pulse, t0=t[36], sigma=0.1)
    rho0 = W.half_filled_rho(h)
    L, R = W.free_triangles(h, rho0, t, n_rows=ns)
    rows = oracle.f_rows_needed(order, ns, n_t)
    Fr = W.free_rhs_rows(h, L, R, rows)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, v, pulse)
    run = kbe.Run(ctx)
    run.L[: len(L)].copy_(_dev(L))
    run.R[: len(R)].copy_(_dev(R))
    for j in rows:
        run.F[j % kbe.KBE_RING_ROWS, :, : j + 1].copy_(_dev(Fr[j]))
    for n in range(ns, n_t):
        run.step(n, P=2)
    ctx.sync_status()
    Lf = np.zeros((W.tri_size(n_t), M, M), np.complex128)
    Rf = np.zeros_like(Lf)
    Lf[: len(L)], Rf[: len(R)] = L, R
    Lo, Ro, _ = oracle.run(t, order, h, U, v, pulse, 2, Lf, Rf, Fr, ns, n_t, nthreads=oracle.threads_available())
    Lg = run.L[: W.tri_size(n_t)].cpu().numpy()
    Rg = run.R[: W.tri_size(n_t)].cpu().numpy()
    assert _rel(Lg, Lo) < TOL and _rel(Rg, Ro) < TOL
    del torch


def test_errors_are_reported_not_raised_on_device(kbe):
    import torch
    M, n_t = 2, 10
    t, order, h, rho0, U, L, R = _case(M, n_t, 1)
    ctx = kbe.Context(M, n_t)
    Ld, Rd = _dev(L), _dev(R)
    Sl = torch.zeros((n_t, M, M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    out = torch.zeros((2, n_t, M, M), dtype=torch.complex128, device="cuda")
    with pytest.raises(kbe.KBEError) as e:  # no grid yet
        ctx.history_slice(3, Ld, Rd, Sl, Sg, out)
    assert e.value.status == kbe.KBE_ESTATE
    ctx.set_grid(t, order)
    with pytest.raises(kbe.KBEError) as e:  # no model yet
        ctx.selfenergy_slice(3, Ld, Rd, Sl, Sg)
    assert e.value.status == kbe.KBE_ESTATE
    ctx.set_model(h, U, W.site_potential(M), None)
    with pytest.raises(kbe.KBEError) as e:
        ctx.history_slice(n_t, Ld, Rd, Sl, Sg, out)
    assert e.value.status == kbe.KBE_ERANGE
    # a misaligned device pointer is rejected before any launch
    lib = kbe.lib()
    import ctypes
    st = lib.kbe_history_slice(ctx._h, 3, 0, ctypes.c_void_p(Ld.data_ptr() + 8), ctypes.c_void_p(Rd.data_ptr()),
                               ctypes.c_void_p(Sl.data_ptr()), ctypes.c_void_p(Sg.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()), None)
    assert st == kbe.KBE_EINVAL
    # a non-finite input is reported through the status word
    Lbad = L.copy()
    Lbad[W.tri_index(3, 1), 0, 1] = np.nan
    ctx.selfenergy_slice(3, _dev(Lbad), Rd, Sl, Sg)
    with pytest.raises(kbe.KBEError) as e:
        ctx.sync_status()
    assert e.value.status == kbe.KBE_ENUMERIC
    ctx.sync_status()  # cleared
    ctx.selfenergy_slice(3, Ld, Rd, Sl, Sg)  # the context stays usable
    ctx.history_slice(3, Ld, Rd, Sl, Sg, out)
    ctx.sync_status()


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_row_band_partials_sum_to_the_slice(kbe, world):
    """The per-device share of the one-system split (kbe_history_slice_band):
    the partial slices of the row bands of parallel.row_bands, computed one
    after another on this GPU and summed (the all-reduce of the plan), give
    kbe_history_slice's slice (1e-14) and the oracle's (1e-12); an empty band
    contributes nothing."""
    import torch
    from paper_2405_08737_gb300 import parallel
    M, n_t = 5, 45
    t, order, h, rho0, U, L, R = _case(M, n_t, 17, "free")
    ctx = _ctx(kbe, M, n_t, t, order, h, U)
    Ld, Rd = _dev(L), _dev(R)
    n = n_t - 1
    Sl, Sg = oracle.sigma_row(oracle.local_U4(U), n, L, R)
    Sld, Sgd = _dev(Sl), _dev(Sg)
    full = torch.zeros((2, n + 1, M, M), dtype=torch.complex128, device="cuda")
    ctx.history_slice(n, Ld, Rd, Sld, Sgd, full)
    total = torch.zeros_like(full)
    part = torch.empty_like(full)
    for lo, hi in parallel.row_bands(n + 1, world):
        ctx.history_slice_band(n, lo, hi, Ld, Rd, Sld, Sgd, part)
        total += part
    ctx.history_slice_band(n, 7, 7, Ld, Rd, Sld, Sgd, part)
    ctx.sync_status()
    assert not part.abs().any()
    ref = oracle.history_slice(t, order, n, L, R, Sl, Sg, nthreads=8)
    f, tot = full.cpu().numpy(), total.cpu().numpy()
    assert _rel(tot, f) < 1e-14 and _rel(tot, ref) < TOL
    with pytest.raises(kbe.KBEError) as e:
        ctx.history_slice_band(n, 5, 4, Ld, Rd, Sld, Sgd, part)
    assert e.value.status == kbe.KBE_EINVAL
    ctx.close()


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_step_phases_with_row_bands(kbe, world):
    """The phases of a KBE step (kbe_step_predict, kbe_step_sweep_band,
    kbe_step_sweep_finish) with the slice summed over the row bands of
    `world` ranks, run one after another on this GPU (what
    parallel.sharded_step does with one band per device and an all-reduce):
    with one band the rows are kbe_step's bitwise; with several, within
    1e-13 of them and 1e-12 of the oracle's step."""
    import torch
    from paper_2405_08737_gb300 import parallel
    M, n_t, seed = 4, 41, 12
    t, order = W.grid(n_t, 0.05, 0.4, seed)
    h = W.goe_h(M, seed)
    U, v = np.linspace(0.5, 2.0, M), W.site_potential(M)
    pulse = {"E0": 0.5, "t0": float(t[n_t // 2]), "sigma": 0.4, "omega": 2.0}
    n = n_t - 1
    Lh, Rh, F = W.restart_state(h, W.half_filled_rho(h), t, order, n, n)
    runs = []
    for phased in (False, True):
        ctx = kbe.Context(M, n_t)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, pulse)
        run = kbe.Run(ctx)
        run.L[: W.tri_size(n)] = torch.as_tensor(Lh, device="cuda")
        run.R[: W.tri_size(n)] = torch.as_tensor(Rh, device="cuda")
        for j, Fj in F.items():
            run.F[j % kbe.KBE_RING_ROWS, :, : j + 1] = torch.as_tensor(Fj, device="cuda")
        if not phased:
            run.step(n, P=2)
        else:
            bands = parallel.row_bands(n + 1, world)
            parts = [torch.zeros_like(run.I) for _ in bands]
            ctx.step_predict(n, run.L, run.R, run.F)
            for _ in range(2):
                for (lo, hi), part in zip(bands, parts):
                    ctx.step_sweep_band(n, lo, hi, run.L, run.R, run.Sl, run.Sg, part)
                total = parts[0].clone()
                for part in parts[1:]:
                    total += part
                ctx.step_sweep_finish(n, run.L, run.R, total, run.F)
        ctx.sync_status()
        runs.append(run)
    p = W.tri_size(n)
    a = [r.L[p:p + n + 1].cpu().numpy() for r in runs]
    b = [r.R[p:p + n + 1].cpu().numpy() for r in runs]
    if world == 1:
        assert np.array_equal(a[0], a[1]) and np.array_equal(b[0], b[1])
    else:
        assert _rel(a[1], a[0]) < 1e-13 and _rel(b[1], b[0]) < 1e-13
    L = np.zeros((W.tri_size(n + 1), M, M), np.complex128)
    R = np.zeros_like(L)
    L[:p], R[:p] = Lh, Rh
    Lo, Ro, _ = oracle.run(t, order, h, U, v, pulse, 2, L, R, F, n, n + 1)
    assert _rel(a[1], Lo[p:]) < 1e-12 and _rel(b[1], Ro[p:]) < 1e-12
    for r in runs:
        r.ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "split", "df64"])
def test_run_steps_is_the_step_loop(kbe, precision):
    """kbe_run_steps (the steps of rows n_first..n_last in one call) gives
    bitwise the rows, slices and ring of one kbe_step call per row, also when
    a run continues from a later row; bad row ranges are rejected."""
    import torch
    M, n_t, seed = 3, 37, 14
    t, order = W.grid(n_t, 0.05, 0.4, seed)
    h = W.goe_h(M, seed)
    U, v = np.linspace(0.5, 2.0, M), W.site_potential(M)
    pulse = dict(W.PULSE_CHAIN, t0=float(t[n_t // 2]), sigma=0.3)
    runs = []
    for mode in ("loop", "one call", "two calls"):
        ctx = kbe.Context(M, n_t)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, pulse)
        run = kbe.Run(ctx)
        run.init_uncorrelated(W.half_filled_rho(h))
        if mode == "loop":
            for n in range(1, n_t):
                run.step(n, P=2, precision=precision)
        elif mode == "one call":
            run.run_steps(1, n_t - 1, P=2, precision=precision)
        else:
            run.run_steps(1, 20, P=2, precision=precision)
            run.run_steps(21, n_t - 1, P=2, precision=precision)
        ctx.sync_status()
        runs.append(run)
    for other in runs[1:]:
        for a, b in ((runs[0].L, other.L), (runs[0].R, other.R), (runs[0].F, other.F), (runs[0].I, other.I),
                     (runs[0].Sl, other.Sl), (runs[0].Sg, other.Sg)):
            assert torch.equal(a, b)
    ctx = runs[0].ctx
    for lo, hi in ((0, 5), (5, 4), (1, n_t)):
        with pytest.raises(kbe.KBEError) as e:
            runs[0].run_steps(lo, hi, P=2, precision=precision)
        assert e.value.status in (kbe.KBE_EINVAL, kbe.KBE_ERANGE)
    for r in runs:
        r.ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("M,n_t,launches", [(2, 100, 2), (8, 80, None)])
def test_run_steps_cooperative_rows(kbe, M, n_t, launches):
    """FP64 rows of at most 4096 entries run in one cooperative launch per
    64 rows with device-wide barriers between the phases of a step: the
    dimer's 99 steps take two launches, and a run of an 8-orbital chain
    crosses from those rows (n <= 63) to the per-kernel step; both give
    bitwise the rows, slice and ring of one kbe_step call per row."""
    import torch
    seed = 21
    t, order = W.grid(n_t, 0.05, 0.4, seed)
    h = W.goe_h(M, seed)
    U, v = np.linspace(0.5, 2.0, M), W.site_potential(M)
    pulse = dict(W.PULSE_CHAIN, t0=float(t[n_t // 3]), sigma=0.3)
    runs = []
    for one_call in (False, True):
        ctx = kbe.Context(M, n_t)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, pulse)
        run = kbe.Run(ctx)
        run.init_uncorrelated(W.half_filled_rho(h))
        if one_call:
            run.run_steps(1, n_t - 1, P=2)
            if launches is not None:
                assert ctx.last_launch_count == launches
        else:
            for n in range(1, n_t):
                run.step(n, P=2)
        ctx.sync_status()
        runs.append(run)
    for a, b in ((runs[0].L, runs[1].L), (runs[0].R, runs[1].R), (runs[0].F, runs[1].F), (runs[0].I, runs[1].I),
                 (runs[0].Sl, runs[1].Sl), (runs[0].Sg, runs[1].Sg)):
        assert torch.equal(a, b)
    assert bool(torch.isfinite(runs[1].L).all())
    for r in runs:
        r.ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("barrier", [0, 6, 272, 10**6])
def test_run_barrier_timeout_is_reported_and_the_context_recovers(kbe, barrier):
    """The failure path of the cooperative run launch, with no fault: block
    0 leaves at one device-wide barrier without arriving
    (kbe_debug_withhold_run) and the waits give up after 4096 polls.  The
    launch returns, the status reads KBE_ETIMEOUT, and the next run on the
    same context is bitwise the step loop again; a barrier beyond the launch's
    last (39 steps of two sweeps: 1 + 39 x 7 = 274 barriers) withholds nothing."""
    import torch
    M, n_t, seed = 2, 40, 5
    t, order = W.grid(n_t, 0.05, 0.4, seed)
    h = W.goe_h(M, seed)
    U, v = np.linspace(0.5, 2.0, M), W.site_potential(M)
    rho0 = W.half_filled_rho(h)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, v, None)
    ref = kbe.Run(ctx)
    ref.init_uncorrelated(rho0)
    for n in range(1, n_t):
        ref.step(n, P=2)
    ctx.sync_status()
    run = kbe.Run(ctx)
    run.init_uncorrelated(rho0)
    ctx.debug_withhold_run(barrier, 4096)
    run.run_steps(1, n_t - 1, P=2)
    if barrier < 274:
        with pytest.raises(kbe.KBEError) as e:
            ctx.sync_status()
        assert e.value.status == kbe.KBE_ETIMEOUT
        run.init_uncorrelated(rho0)
        run.run_steps(1, n_t - 1, P=2)
    ctx.sync_status()
    for a, b in ((ref.L, run.L), (ref.R, run.R), (ref.F, run.F), (ref.I, run.I), (ref.Sl, run.Sl), (ref.Sg, run.Sg)):
        assert torch.equal(a, b)
    with pytest.raises(kbe.KBEError):
        ctx.debug_withhold_run(-1, 4096)
    ctx.close()


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["P1", "P3", "dense", "adaptive", "profiling"])
def test_run_steps_other_settings(kbe, mode):
    """kbe_run_steps is bitwise the step loop with one and three sweeps per
    step (the cooperative kernel), and with the settings under which it keeps
    the per-kernel step: a dense interaction, adaptive history orders (the
    chosen orders equal too) and profiling."""
    import torch
    M, n_t, seed = 2, 30, 8
    P = {"P1": 1, "P3": 3}.get(mode, 2)
    t, order = W.grid(n_t, 0.05, 0.4, seed)
    h = W.goe_h(M, seed)
    U, v = np.linspace(0.5, 2.0, M), W.site_potential(M)
    pulse = dict(W.PULSE_CHAIN, t0=float(t[n_t // 2]), sigma=0.3)
    runs = []
    for one_call in (False, True):
        ctx = kbe.Context(M, n_t)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, pulse)
        if mode == "dense":
            ctx.set_interaction(W.coulomb_tensor(M, 2, U=1.3))
        elif mode == "adaptive":
            ctx.set_adaptive_orders(4)
        elif mode == "profiling":
            ctx.set_profiling(True)
        run = kbe.Run(ctx)
        run.init_uncorrelated(W.half_filled_rho(h))
        if one_call:
            run.run_steps(1, n_t - 1, P=P)
        else:
            for n in range(1, n_t):
                run.step(n, P=P)
        ctx.sync_status()
        runs.append(run)
    for a, b in ((runs[0].L, runs[1].L), (runs[0].R, runs[1].R), (runs[0].F, runs[1].F), (runs[0].I, runs[1].I),
                 (runs[0].Sl, runs[1].Sl), (runs[0].Sg, runs[1].Sg)):
        assert torch.equal(a, b)
    if mode == "adaptive":
        assert np.array_equal(runs[0].ctx.history_orders(n_t), runs[1].ctx.history_orders(n_t))
    if mode == "profiling":
        k, ms = runs[1].ctx.read_profiling()
        assert k >= (n_t - 1) * P and ms > 0  # one record per sweep's contraction (and the start row's)
    for r in runs:
        r.ctx.close()
